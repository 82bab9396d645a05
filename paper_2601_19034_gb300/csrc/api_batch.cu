// C ABI of the batched force call (include/qnep.h, "Batched evaluation"): the batch
// description (structures, boxes, k-tables, work items), its workspaces, the launch
// sequence and the autotuner that picks the block shape and the item order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <array>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qnep.h"
#include "batch_internal.cuh"
#include "kset_host.h"

using namespace qnep;

static_assert((int)QNEP_BATCH_CONTRACT_FP32 == (int)BATCH_CONTRACT_FP32 &&
                  (int)QNEP_BATCH_CONTRACT_BF16X3 == (int)BATCH_CONTRACT_BF16X3,
              "contraction codes of the C ABI and of the kernels agree");
static_assert((int)QNEP_BATCH_CONTRACT_BF16 == (int)BATCH_CONTRACT_BF16, "contraction codes agree");

struct qnep_batch {
    qnep_hparams hp{};
    qnep_elec es{};
    ParamLayout lay{};
    int n_cand = 0, n_groups = 0;
    float* d_pt = nullptr;                  // [group][p][CG]
    int cap_l_user = 0, cap_a_user = 0;
    int warps = 8;                          // warps per block of the item kernel (4 or 8)
    int order_policy = QNEP_BATCH_ORDER_LARGEST_FIRST;
    int contract = QNEP_BATCH_CONTRACT_FP32;   // descriptor contraction: FP32 FMAs or tensor cores
    int num_sms = 152;
    // batch description (rebuilt when the structures or boxes change)
    bool have_desc = false;
    // static geometry (training on fixed structures): the candidate-independent pre-pass is kept
    // from the call that built it while the description, the input pointers and the operand
    // images it needs are the same and the caller has not reported a change
    bool static_geom = false, geom_valid = false, geom_tc = false;
    const float* geom_pos = nullptr;
    const int* geom_types = nullptr;
    int n_struct = 0, n_total = 0, nmax = 0, nph_max = 0, nk_max = 0;
    bool has_empty = false;                 // a structure without atoms (its energy is written as 0)
    std::vector<int> h_off;
    std::vector<double> h_box;
    int cap_l = 0, cap_a = 0;
    std::vector<int2> items_lpt, items_nat;
    BatchStruct* d_st = nullptr;
    BatchKTab* d_kt = nullptr;
    BatchKTri* d_ktri = nullptr;          // general-cell phase data per k-table (pre-pass)
    float* d_rot = nullptr;               // per structure: rotation into the restricted cell form, flag
    int4* d_chunk = nullptr;
    float4* d_kvec = nullptr;
    int* d_kreal = nullptr;
    int2* d_items_lpt = nullptr;
    int2* d_items_nat = nullptr;
    int n_items = 0;
    // pre-pass outputs (element counts allocated)
    struct {
        size_t spos4 = 0, sidx = 0, order = 0, spec = 0, cells = 0, list = 0, ang = 0, cnt_list = 0, cnt_ang = 0,
               phase = 0, geo_rad = 0, geo_ang = 0, bsum = 0, bimg = 0, zsum = 0;
    } alloc;
    float4* spos4 = nullptr;
    int* sidx = nullptr;
    int* order = nullptr;
    int* spec_off = nullptr;
    int* cell_start = nullptr;
    int* nbr_list = nullptr;
    int* cnt_list = nullptr;
    int* nbr_ang = nullptr;
    int* cnt_ang = nullptr;
    float2* phase = nullptr;
    float* geo_rad = nullptr;
    float* geo_ang = nullptr;
    float* bsum = nullptr;
    unsigned char* bimg = nullptr;          // B^A operand images (tensor-core contraction only)
    float4* zsum = nullptr;                 // per-slot BEC accumulators (calls with BEC only)
    // per-slot scratch
    size_t slot_bytes_alloc = 0;
    int slots_alloc = 0;
    BatchScratch sc{};
    float* scratch = nullptr;
    unsigned int* d_work = nullptr;
    unsigned int* d_status = nullptr;       // [0] this call's kernels, [1] the pre-pass that built the
                                            // lists in use (kept, with them, while static geometry is reused)
    cudaStream_t last_stream = nullptr;
    std::map<std::tuple<int, int, int, int>, int> per_sm_cache;   // (warps, nph_max, contract, 0 | virial 1 | BEC 2) -> blocks per SM
    // host-buffer entry point: device copies of the inputs and outputs (grown on demand)
    float* io_pos = nullptr;
    int* io_types = nullptr;
    double* io_energy = nullptr;
    float* io_forces = nullptr;
    float* io_charges = nullptr;
    double* io_virial = nullptr;
    float* io_bec = nullptr;
    double* io_qtot = nullptr;
    double* io_pol = nullptr;
    size_t io_atoms = 0, io_evals = 0, io_pairs = 0;
    // stage timers: events around the pre-pass and the item kernel of each profiled call
    bool profiling = false, pending = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    double stage_ms[2] = {0.0, 0.0};
    int timed_calls = 0;
    std::string err;
};

namespace {

qnep_status failb(qnep_batch* b, qnep_status s, const std::string& msg) {
    if (b) b->err = msg;
    return s;
}

#define CKB(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return failb(b, e_ == cudaErrorMemoryAllocation ? QNEP_ERR_OOM : QNEP_ERR_CUDA,        \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

template <class T>
cudaError_t regrow(T** p, size_t count, size_t* have) {
    if (count <= *have && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
    if (e == cudaSuccess) *have = count;
    return e;
}

template <class T>
cudaError_t upload(T** p, const std::vector<T>& v) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

float list_cutoff_b(const qnep_batch* b) {
    float rc = b->hp.rc_radial;
    if (b->es.mode == 1 && (float)b->es.rc_real > rc) rc = (float)b->es.rc_real;
    return rc;
}

// Structures, boxes, k-tables and work items of a new batch description.
qnep_status describe(qnep_batch* b, int n_struct, const int* off, const double* boxes, cudaStream_t st) {
    const float rcl = list_cutoff_b(b);
    std::vector<BatchStruct> sts(n_struct);
    std::vector<BatchKTab> kts;
    std::vector<BatchKTri> ktris;
    std::vector<int4> chunks;
    std::vector<int> kreal;
    std::vector<float4> kvec;
    std::map<std::array<double, 9>, int> tab_of;
    std::vector<int> nk_of;   // padded k count per table
    int cell_total = 0, nmax = 0, nph_max = 0, nk_max = 0;
    double dens_max = 0.0;
    const double two_pi = 6.283185307179586, ke = 14.3996454784;
    std::vector<float> rot((size_t)n_struct * 12, 0.f);   // per structure: R (row-major), flag, pad
    for (int s = 0; s < n_struct; ++s) {
        const double* bx0 = boxes + 9 * (size_t)s;
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(bx0[k])) return failb(b, QNEP_ERR_ARG, "box has a non-finite entry");
        // orthorhombic, or a general cell in the restricted form a = (a_x, 0, 0), b = (b_x, b_y, 0),
        // c = (c_x, c_y, c_z) with a_x, b_y, c_z > 0: its H and H^-1 are lower triangular, so the x and
        // y components of k = 2 pi H^-1 n depend on (n1, n2) only, as the k-space field pass assumes
        // for a column of wave vectors.  Any other general cell is rotated into that form (rows of R:
        // e1 = a / |a|, e3 = a x b / |a x b|, e2 = e3 x e1; the pre-pass rotates the positions, the
        // outputs are rotated back)
        double bx[9];
        for (int k = 0; k < 9; ++k) bx[k] = bx0[k];
        float* rs = rot.data() + 12 * (size_t)s;
        rs[0] = rs[4] = rs[8] = 1.f;
        if (bx[1] != 0 || bx[2] != 0 || bx[5] != 0) {
            double R[9];
            if (!rotate_to_restricted(bx0, R, bx)) return failb(b, QNEP_ERR_ARG, "the cell vectors must be independent");
            for (int k = 0; k < 9; ++k) rs[k] = (float)R[k];
            rs[9] = 1.f;
        }
        const bool tri = bx[3] != 0 || bx[6] != 0 || bx[7] != 0 || bx[1] != 0 || bx[2] != 0 || bx[5] != 0;
        if (tri && !(bx[0] > 0 && bx[4] > 0 && bx[8] > 0))
            return failb(b, QNEP_ERR_ARG, "the cell vectors must be right-handed (a_x, b_y, c_z > 0)");
        double hinv[9];
        const double det = invert3(bx, hinv);
        double L[3], width[3];
        for (int d = 0; d < 3; ++d) {
            const double* av = bx + 3 * d;
            L[d] = tri ? std::sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]) : bx[4 * d];
            // perpendicular width V / |a_e x a_f| (the cell grid needs width >= cutoff); the edge if orthorhombic
            const double* e = bx + 3 * ((d + 1) % 3);
            const double* f = bx + 3 * ((d + 2) % 3);
            const double cx = e[1] * f[2] - e[2] * f[1], cy = e[2] * f[0] - e[0] * f[2], cz = e[0] * f[1] - e[1] * f[0];
            width[d] = tri ? det / std::sqrt(cx * cx + cy * cy + cz * cz) : L[d];
        }
        BatchStruct& t = sts[s];
        t.atom_off = off[s];
        t.n = off[s + 1] - off[s];
        if (t.n < 0) return failb(b, QNEP_ERR_ARG, "atom offsets must be non-decreasing");
        if (t.n > 32768) return failb(b, QNEP_ERR_UNSUPPORTED, "batched structures hold at most 32768 atoms");
        nmax = std::max(nmax, t.n);
        Geom& g = t.g;
        g.tri = tri ? 1 : 0;
        for (int k = 0; k < 9; ++k) {
            g.H[k] = (float)bx[k];
            g.Hi[k] = (float)hinv[k];
        }
        g.ncells = 1;
        for (int d = 0; d < 3; ++d) {
            if (!(L[d] > 0)) return failb(b, QNEP_ERR_ARG, "box edge must be positive");
            if (width[d] < rcl) return failb(b, QNEP_ERR_UNSUPPORTED, "cell width shorter than the list cutoff");
            g.L[d] = (float)L[d];
            g.invL[d] = (float)(1.0 / L[d]);
            int nc = (int)std::floor(width[d] / rcl);
            g.nc[d] = std::min(std::max(nc, 1), 8);
            g.ncells *= g.nc[d];
        }
        g.rc_list = rcl;
        g.rc_radial = b->hp.rc_radial;
        g.rc_angular = b->hp.rc_angular;
        g.rc_real = b->es.mode == 1 ? (float)b->es.rc_real : 0.f;
        g.list_sa = g.list_se = g.ang_sa = g.ang_se = 0;
        t.cell_off = cell_total;
        cell_total += g.ncells + 1;
        dens_max = std::max(dens_max, t.n / std::fabs(det));
        std::array<double, 9> key;
        for (int k = 0; k < 9; ++k) key[k] = bx[k];
        auto it = tab_of.find(key);
        if (it == tab_of.end()) {
            // the phase-factor count is known from n_max alone: refuse before enumerating the k-set
            if (kset_phase_count(L, b->es.kmax) > BATCH_MAX_NPH)
                return failb(b, QNEP_ERR_UNSUPPORTED, "box too large for the batched k-space tables");
            KSet ks = tri ? build_kset_box(bx, b->es.kmax, b->es.alpha) : build_kset(L, b->es.kmax, b->es.alpha);
            BatchKTab kt{};
            kt.n1max = ks.nmax[0];
            kt.n2max = ks.nmax[1];
            kt.n3max = ks.nmax[2];
            kt.yoff = kt.n1max + 1;
            kt.zoff = kt.yoff + 2 * kt.n2max + 1;
            kt.nph = kt.zoff + 2 * kt.n3max + 8;
            if (kt.nph > BATCH_MAX_NPH)
                return failb(b, QNEP_ERR_UNSUPPORTED, "box too large for the batched k-space tables");
            kt.nchunk = (int)ks.chunk_col.size();
            kt.chunk_off = (int)chunks.size();
            for (int d = 0; d < 3; ++d) {
                double il = 1.0 / L[d];
                kt.invl_hi[d] = (float)il;
                kt.invl_lo[d] = (float)(il - (double)kt.invl_hi[d]);
            }
            BatchKTri kr{};
            kr.tri = tri ? 1 : 0;
            for (int k = 0; k < 9; ++k) {
                kr.hi_hi[k] = (float)hinv[k];
                kr.hi_lo[k] = (float)(hinv[k] - (double)kr.hi_hi[k]);
            }
            kt.kreal_off = (int)kreal.size();
            for (int h = 0; h < kt.nchunk; ++h) {
                const int4& c = ks.cols[ks.chunk_col[h]];
                const int n3 = c.z + (8 * h - c.w);
                int cnt = 0;   // the column's entries are contiguous from the chunk start
                for (int q = 0; q < 8; ++q)
                    if (ks.kg[8 * h + q] > 0.f) {
                        kreal.push_back(8 * h + q);
                        ++cnt;
                    }
                chunks.push_back(make_int4(c.x, c.y, n3, cnt));
                for (int q = 0; q < 8; ++q) {
                    const float gk = ks.kg[8 * h + q];
                    if (tri) {   // k_d = 2 pi sum_c H^-1[d][c] n_c
                        const double nv[3] = {(double)c.x, (double)c.y, (double)(n3 + q)};
                        double kd[3];
                        for (int d = 0; d < 3; ++d)
                            kd[d] = two_pi * (hinv[3 * d] * nv[0] + hinv[3 * d + 1] * nv[1] + hinv[3 * d + 2] * nv[2]);
                        kvec.push_back(make_float4((float)kd[0], (float)kd[1], (float)kd[2], (float)(4.0 * ke * gk)));
                    } else {
                        kvec.push_back(make_float4((float)(two_pi * c.x / L[0]), (float)(two_pi * c.y / L[1]),
                                                   (float)(two_pi * (n3 + q) / L[2]), (float)(4.0 * ke * gk)));
                    }
                }
            }
            kt.nkr = (int)kreal.size() - kt.kreal_off;
            nph_max = std::max(nph_max, kt.nph);
            nk_max = std::max(nk_max, 8 * kt.nchunk);
            it = tab_of.emplace(key, (int)kts.size()).first;
            kts.push_back(kt);
            ktris.push_back(kr);
            nk_of.push_back(8 * kt.nchunk);
        }
        t.ktab = it->second;
    }
    nph_max += nph_max & 1;   // even: every atom's phase row starts on a 16-byte boundary (bulk copies)
    // neighbour capacities from the densest structure (2x the mean count + margin)
    const double pi43 = 4.18879020478639;
    int cl = b->cap_l_user, ca = b->cap_a_user;
    if (cl <= 0) cl = ((int)(2.0 * pi43 * rcl * rcl * rcl * dens_max) + 32 + 31) / 32 * 32;
    if (ca <= 0) {
        double ra = b->hp.rc_angular;
        ca = ((int)(2.0 * pi43 * ra * ra * ra * dens_max) + 16 + 15) / 16 * 16;
    }
    // work items: (structure, group); cost ~ atoms x (descriptor work + wave vectors)
    std::vector<std::pair<double, int2>> it;
    b->has_empty = false;
    for (int s = 0; s < n_struct; ++s) {
        if (sts[s].n == 0) {
            b->has_empty = true;
            continue;
        }
        const double cost = (double)sts[s].n * (2800.0 + nk_of[sts[s].ktab]);
        for (int gi = 0; gi < b->n_groups; ++gi) it.push_back({cost, make_int2(s, gi)});
    }
    b->items_nat.clear();
    for (auto& x : it) b->items_nat.push_back(x.second);
    std::stable_sort(it.begin(), it.end(), [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) {
        return x.first > y.first;
    });
    b->items_lpt.clear();
    for (auto& x : it) b->items_lpt.push_back(x.second);
    // uploads (in-flight work of the previous description may still read the old tables)
    if (b->have_desc && b->last_stream) CKB(cudaStreamSynchronize(b->last_stream));
    CKB(cudaStreamSynchronize(st));
    CKB(upload(&b->d_st, sts));
    CKB(upload(&b->d_kt, kts));
    CKB(upload(&b->d_ktri, ktris));
    CKB(upload(&b->d_rot, rot));
    CKB(upload(&b->d_chunk, chunks));
    CKB(upload(&b->d_kvec, kvec));
    CKB(upload(&b->d_kreal, kreal));
    CKB(upload(&b->d_items_lpt, b->items_lpt));
    CKB(upload(&b->d_items_nat, b->items_nat));
    b->n_items = (int)b->items_lpt.size();
    b->n_struct = n_struct;
    b->n_total = off[n_struct];
    b->nmax = nmax;
    b->nph_max = nph_max;
    b->nk_max = nk_max;
    b->cap_l = cl;
    b->cap_a = ca;
    const size_t N = (size_t)b->n_total, S = (size_t)b->hp.n_species;
    CKB(regrow(&b->spos4, N, &b->alloc.spos4));
    CKB(regrow(&b->sidx, N, &b->alloc.sidx));
    CKB(regrow(&b->order, N, &b->alloc.order));
    CKB(regrow(&b->spec_off, (size_t)n_struct * (MAX_SPECIES + 1), &b->alloc.spec));
    CKB(regrow(&b->cell_start, (size_t)cell_total, &b->alloc.cells));
    CKB(regrow(&b->nbr_list, N * (size_t)cl, &b->alloc.list));
    CKB(regrow(&b->nbr_ang, N * (size_t)ca, &b->alloc.ang));
    CKB(regrow(&b->cnt_list, N * S, &b->alloc.cnt_list));
    CKB(regrow(&b->cnt_ang, N * S, &b->alloc.cnt_ang));
    CKB(regrow(&b->phase, N * (size_t)batch_phase_stride(nph_max), &b->alloc.phase));
    CKB(regrow(&b->geo_rad, N * (size_t)cl * BATCH_GR, &b->alloc.geo_rad));
    CKB(regrow(&b->geo_ang, N * (size_t)ca * BATCH_GA, &b->alloc.geo_ang));
    CKB(regrow(&b->bsum, N * (size_t)batch_bstride(b->hp.n_species), &b->alloc.bsum));
    if (batch_contract_tc(b->contract)) CKB(regrow(&b->bimg, N * (size_t)BIMG_BYTES, &b->alloc.bimg));
    b->h_off.assign(off, off + n_struct + 1);
    b->h_box.assign(boxes, boxes + 9 * (size_t)n_struct);
    b->have_desc = true;
    b->geom_valid = false;   // new tables and lists: the next call runs the pre-pass
    return QNEP_OK;
}

// Per-slot scratch for the current description and block shape.
qnep_status ensure_scratch(qnep_batch* b, int slots, bool bec, cudaStream_t st) {
    const size_t nm = (size_t)std::max(b->nmax, 1), nk = (size_t)std::max(b->nk_max, 8);
    BatchScratch& sc = b->sc;
    const size_t sA = nm * NANG * CG, sD = nm * 2 * NDES * CG, sN = nm * CG, sK = nk * CG;
    const size_t sP = (size_t)((nm + 511) / 512) * sK;   // partial structure factors per 512 atoms
    // floats per slot: A, duq, uq (2), qc (1), fk/fr/fsum (4 each), sk (2), skp (2), virial sums
    // (8 warps x 9 x CG doubles)
    const size_t sV = (size_t)8 * 9 * CG;
    // (8 warps x 9 x CG doubles)
    const size_t per = sA + sD + 2 * sN + sN + 12 * sN + 2 * sK + 2 * sP + 2 * sV + 64;
    const size_t bytes = per * sizeof(float) * (size_t)slots;
    if (bytes > b->slot_bytes_alloc || !b->scratch) {
        CKB(cudaStreamSynchronize(st));
        if (b->last_stream) CKB(cudaStreamSynchronize(b->last_stream));
        if (b->scratch) cudaFree(b->scratch);
        b->scratch = nullptr;
        b->slot_bytes_alloc = 0;
        CKB(cudaMalloc((void**)&b->scratch, bytes));
        b->slot_bytes_alloc = bytes;
    }
    // carve: arrays of all slots back to back (each 16-byte aligned)
    float* p = b->scratch;
    auto take = [&](size_t floats) {
        float* q = p;
        p += (floats + 3) & ~(size_t)3;
        return q;
    };
    sc.stride_A = sA;
    sc.stride_duq = sD;
    sc.stride_n = sN;
    sc.stride_k = sK;
    sc.A = take(sA * slots);
    sc.duq = take(sD * slots);
    sc.uq = reinterpret_cast<float2*>(take(2 * sN * slots));
    sc.qc = take(sN * slots);
    sc.fk = reinterpret_cast<float4*>(take(4 * sN * slots));
    sc.fr = reinterpret_cast<float4*>(take(4 * sN * slots));
    sc.fsum = reinterpret_cast<float4*>(take(4 * sN * slots));
    sc.sk = reinterpret_cast<float2*>(take(2 * sK * slots));
    sc.stride_p = sP;
    sc.skp = reinterpret_cast<float2*>(take(2 * sP * slots));
    sc.vir = reinterpret_cast<double*>(take(2 * sV * slots));
    b->slots_alloc = slots;
    // BEC accumulators (three float4 per atom and candidate) in a buffer of their own: asking for BEC
    // never moves the scratch above, which graphs captured from calls without BEC keep using
    sc.zsum = nullptr;
    if (bec) {
        const size_t nz = 3 * sN * (size_t)slots;
        if (nz > b->alloc.zsum) {
            CKB(cudaStreamSynchronize(st));
            if (b->last_stream) CKB(cudaStreamSynchronize(b->last_stream));
        }
        CKB(regrow(&b->zsum, nz, &b->alloc.zsum));
        sc.zsum = b->zsum;
    }
    return QNEP_OK;
}

bool same_desc(const qnep_batch* b, int n_struct, const int* off, const double* boxes) {
    if (!b->have_desc || b->n_struct != n_struct) return false;
    if (std::memcmp(b->h_off.data(), off, sizeof(int) * (n_struct + 1)) != 0) return false;
    return std::memcmp(b->h_box.data(), boxes, sizeof(double) * 9 * (size_t)n_struct) == 0;
}

}  // namespace

namespace {

// Candidate-major parameters [C][P] into the lane-minor layout [group][p][CG] through a
// 32 x 32 shared-memory tile (coalesced reads along p, coalesced writes along the lanes).
__global__ void k_set_params(const float* __restrict__ src, float* __restrict__ dst, int n_cand, int n_par) {
    __shared__ float tile[CG][CG + 1];
    const int g = blockIdx.y, p0 = blockIdx.x * CG;
    for (int r = threadIdx.y; r < CG; r += blockDim.y) {
        const int c = g * CG + r, p = p0 + threadIdx.x;
        if (c < n_cand && p < n_par) tile[r][threadIdx.x] = src[(size_t)c * n_par + p];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < CG; r += blockDim.y) {
        const int p = p0 + r, lane = threadIdx.x, c = g * CG + lane;
        if (c < n_cand && p < n_par) dst[((size_t)g * n_par + p) * CG + lane] = tile[lane][r];
    }
}

}  // namespace

extern "C" {

qnep_status qnep_batch_create(qnep_batch** out, const qnep_hparams* hp, const float* params_host, size_t n_params,
                              int n_candidates, const qnep_elec* es) {
    qnep_batch* b = nullptr;
    if (!out || !hp || !params_host || !es || n_candidates < 1) return QNEP_ERR_ARG;
    *out = nullptr;
    if (hp->n_radial != NR || hp->n_angular != NA || hp->basis_radial != KR || hp->basis_angular != KA ||
        hp->l_max != LMAX || hp->use_4body != 1 || hp->n_neurons != NNEU || hp->n_species < 1 ||
        hp->n_species > MAX_SPECIES)
        return QNEP_ERR_UNSUPPORTED;
    if (!(hp->rc_radial > 0) || !(hp->rc_angular > 0) || hp->rc_angular > hp->rc_radial) return QNEP_ERR_ARG;
    const size_t per = qnep_param_count(hp);
    if (n_params != per * (size_t)n_candidates) return QNEP_ERR_ARG;
    if (es->mode != 1 && es->mode != 2) return QNEP_ERR_UNSUPPORTED;
    if (es->kind != QNEP_EWALD) return QNEP_ERR_UNSUPPORTED;
    if (!(es->alpha > 0) || !(es->kmax > 0) || !std::isfinite(es->alpha) || !std::isfinite(es->kmax))
        return QNEP_ERR_ARG;
    if (es->mode == 1 && (!(es->rc_real > 0) || es->rc_real > hp->rc_radial)) return QNEP_ERR_UNSUPPORTED;
    for (size_t k = 0; k < n_params; ++k)
        if (!std::isfinite(params_host[k])) return QNEP_ERR_ARG;
    std::vector<float> pt;
    try {   // host memory: no exception crosses the C ABI
        b = new qnep_batch();
        b->hp = *hp;
        b->es = *es;
        b->lay = make_layout(hp->n_species);
        b->n_cand = n_candidates;
        b->n_groups = (n_candidates + CG - 1) / CG;
        pt.assign((size_t)b->n_groups * (size_t)b->lay.total * CG, 0.f);
    } catch (const std::bad_alloc&) {
        delete b;
        return QNEP_ERR_OOM;
    }
    const size_t P = (size_t)b->lay.total;
    for (int gi = 0; gi < b->n_groups; ++gi)
        for (int l = 0; l < CG; ++l) {
            const int c = gi * CG + l;
            float* dst = pt.data() + (size_t)gi * P * CG + l;
            if (c < n_candidates) {
                for (size_t p = 0; p < P; ++p) dst[p * CG] = params_host[(size_t)c * P + p];
            } else {
                dst[(size_t)b->lay.sqrt_eps * CG] = 1.f;   // padding lanes: zero network, finite charges
            }
        }
    if (cudaMalloc((void**)&b->d_pt, sizeof(float) * pt.size()) != cudaSuccess ||
        cudaMemcpy(b->d_pt, pt.data(), sizeof(float) * pt.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc((void**)&b->d_work, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_status, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(b->d_status, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
        qnep_batch_destroy(b);
        return QNEP_ERR_CUDA;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        b->num_sms = sms;
    *out = b;
    return QNEP_OK;
}

qnep_status qnep_batch_set_capacity(qnep_batch* b, int cap_list, int cap_angular) {
    if (!b || cap_list < 0 || cap_angular < 0) return QNEP_ERR_ARG;
    b->cap_l_user = cap_list;
    b->cap_a_user = cap_angular;
    b->have_desc = false;   // rebuilt (and lists re-sized) by the next call
    return QNEP_OK;
}

qnep_status qnep_batch_capacity(const qnep_batch* b, int* cap_list, int* cap_angular) {
    if (!b || !cap_list || !cap_angular) return QNEP_ERR_ARG;
    *cap_list = b->cap_l;
    *cap_angular = b->cap_a;
    return QNEP_OK;
}

qnep_status qnep_batch_set_config(qnep_batch* b, int warps, int order) {
    if (!b || (warps != 4 && warps != 8) ||
        (order != QNEP_BATCH_ORDER_LARGEST_FIRST && order != QNEP_BATCH_ORDER_STRUCTURE))
        return QNEP_ERR_ARG;
    b->warps = warps;
    b->order_policy = order;
    return QNEP_OK;
}

qnep_status qnep_batch_set_static_geometry(qnep_batch* b, int enable) {
    if (!b || (enable != 0 && enable != 1)) return QNEP_ERR_ARG;
    b->static_geom = enable != 0;
    b->geom_valid = false;   // the first call after this builds the geometry it keeps
    return QNEP_OK;
}

qnep_status qnep_batch_geometry_changed(qnep_batch* b) {
    if (!b) return QNEP_ERR_ARG;
    b->geom_valid = false;
    return QNEP_OK;
}

qnep_status qnep_batch_set_contraction(qnep_batch* b, int contract) {
    if (!b || (contract != QNEP_BATCH_CONTRACT_FP32 && contract != QNEP_BATCH_CONTRACT_BF16X3 &&
               contract != QNEP_BATCH_CONTRACT_BF16))
        return QNEP_ERR_ARG;
    b->contract = contract;
    if (batch_contract_tc(contract)) b->warps = 8;   // the tensor-core form runs 8 warps
    return QNEP_OK;
}

qnep_status qnep_batch_get_contraction(const qnep_batch* b, int* contract) {
    if (!b || !contract) return QNEP_ERR_ARG;
    *contract = b->contract;
    return QNEP_OK;
}

qnep_status qnep_batch_get_config(const qnep_batch* b, int* warps, int* order) {
    if (!b || !warps || !order) return QNEP_ERR_ARG;
    *warps = b->warps;
    *order = b->order_policy;
    return QNEP_OK;
}

qnep_status qnep_batch_compute(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions,
                               const int* types, const double* boxes, void* stream, double* energy, float* forces,
                               float* charges) {
    qnep_batch_outputs o{energy, forces, charges, nullptr};
    return qnep_batch_compute_outputs(b, n_struct, atom_offsets, positions, types, boxes, stream, &o);
}

qnep_status qnep_batch_compute_outputs(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions,
                                       const int* types, const double* boxes, void* stream,
                                       const qnep_batch_outputs* out) {
    if (!b) return QNEP_ERR_ARG;
    if (!out) return failb(b, QNEP_ERR_ARG, "outputs are NULL");
    double* energy = out->energy;
    float* forces = out->forces;
    float* charges = out->charges;
    double* virial = out->virial;
    const bool bec = out->bec != nullptr;
    if (n_struct < 1 || !atom_offsets || !boxes || !energy) return failb(b, QNEP_ERR_ARG, "bad batch arguments");
    if (atom_offsets[0] != 0) return failb(b, QNEP_ERR_ARG, "atom_offsets[0] must be 0");
    if (atom_offsets[n_struct] > 0 && (!positions || !types))
        return failb(b, QNEP_ERR_ARG, "positions and types are required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!same_desc(b, n_struct, atom_offsets, boxes)) {
        qnep_status s;
        try {
            s = describe(b, n_struct, atom_offsets, boxes, st);
        } catch (const std::bad_alloc&) {   // host tables: no exception crosses the C ABI
            s = failb(b, QNEP_ERR_OOM, "host memory for the batch description could not be obtained");
        }
        if (s != QNEP_OK) {
            b->have_desc = false;
            return s;
        }
    }
    // blocks per SM of this shape (cached: no CUDA calls beyond launches once the batch is known,
    // so the call can be captured in a graph)
    const auto key = std::make_tuple(b->warps, b->nph_max, b->contract, bec ? 2 : (virial ? 1 : 0));
    auto hit = b->per_sm_cache.find(key);
    if (hit == b->per_sm_cache.end())
        hit = b->per_sm_cache
                  .emplace(key, batch_item_blocks_per_sm(b->warps, b->nph_max, b->contract, virial != nullptr, bec))
                  .first;
    const int per_sm = hit->second;
    if (per_sm <= 0) return failb(b, QNEP_ERR_UNSUPPORTED, "item kernel does not fit on an SM");
    const bool tc = batch_contract_tc(b->contract);
    if (tc && (!b->bimg || b->alloc.bimg < (size_t)b->n_total * BIMG_BYTES)) {
        CKB(cudaStreamSynchronize(st));
        CKB(regrow(&b->bimg, (size_t)std::max(b->n_total, 1) * BIMG_BYTES, &b->alloc.bimg));
    }
    const int slots = per_sm * b->num_sms;
    qnep_status s = ensure_scratch(b, slots, bec, st);
    if (s != QNEP_OK) return s;
    // (the tensor-core form's pre-pass writes the B^A operand images instead of the FP32 B^A sums:
    // a change of contraction family rebuilds)
    const bool reuse = b->static_geom && b->geom_valid && b->geom_pos == positions && b->geom_types == types &&
                       b->geom_tc == tc;
    CKB(cudaMemsetAsync(b->d_work, 0, sizeof(unsigned int), st));
    // a reused pre-pass keeps its status word: an overflow it recorded is reported by every call
    // that reads its lists
    CKB(cudaMemsetAsync(b->d_status, 0, (reuse ? 1 : 2) * sizeof(unsigned int), st));
    if (b->has_empty) {   // structures without atoms have no item: their energies (and virials) are zero
        CKB(cudaMemsetAsync(energy, 0, sizeof(double) * (size_t)b->n_cand * n_struct, st));
        if (virial) CKB(cudaMemsetAsync(virial, 0, sizeof(double) * 9 * (size_t)b->n_cand * n_struct, st));
        if (out->total_charge)
            CKB(cudaMemsetAsync(out->total_charge, 0, sizeof(double) * (size_t)b->n_cand * n_struct, st));
        if (out->polarization)
            CKB(cudaMemsetAsync(out->polarization, 0, sizeof(double) * 3 * (size_t)b->n_cand * n_struct, st));
    }
    if (b->profiling) {
        if (b->pending) {   // previous profiled call: harvest its events
            CKB(cudaEventSynchronize(b->ev[2]));
            float t0 = 0.f, t1 = 0.f;
            cudaEventElapsedTime(&t0, b->ev[0], b->ev[1]);
            cudaEventElapsedTime(&t1, b->ev[1], b->ev[2]);
            b->stage_ms[0] += t0;
            b->stage_ms[1] += t1;
            ++b->timed_calls;
        }
        CKB(cudaEventRecord(b->ev[0], st));
    }
    if (!reuse) {
        launch_batch_prep(positions, types, n_struct, b->nmax, b->hp.n_species, b->d_st, b->d_kt, b->d_ktri,
                          b->cell_start, b->spos4, b->sidx, b->order, b->spec_off, b->cap_l, b->cap_a, b->nbr_list,
                          b->cnt_list, b->nbr_ang, b->cnt_ang, b->phase, batch_phase_stride(b->nph_max), b->geo_rad,
                          b->geo_ang, b->bsum, batch_bstride(b->hp.n_species), tc ? b->bimg : nullptr,
                          (float)b->es.alpha, b->d_rot, b->d_status + 1, st);
        b->geom_valid = true;
        b->geom_pos = positions;
        b->geom_types = types;
        b->geom_tc = tc;
    }
    BatchArgs a{};
    a.spos4 = b->spos4;
    a.sidx = b->sidx;
    a.order = b->order;
    a.spec_off = b->spec_off;
    a.nbr_list = b->nbr_list;
    a.cnt_list = b->cnt_list;
    a.nbr_ang = b->nbr_ang;
    a.cnt_ang = b->cnt_ang;
    a.cap_l = b->cap_l;
    a.cap_a = b->cap_a;
    a.phase = b->phase;
    a.nph_stride = batch_phase_stride(b->nph_max);
    a.geo_rad = b->geo_rad;
    a.geo_ang = b->geo_ang;
    a.bsum = b->bsum;
    a.bimg = tc ? b->bimg : nullptr;
    a.bstride = batch_bstride(b->hp.n_species);
    a.st = b->d_st;
    a.kt = b->d_kt;
    a.chunk = b->d_chunk;
    a.kvec = b->d_kvec;
    a.kreal = b->d_kreal;
    a.pt = b->d_pt;
    a.lay = b->lay;
    a.n_cand = b->n_cand;
    a.items = b->order_policy == QNEP_BATCH_ORDER_STRUCTURE ? b->d_items_nat : b->d_items_lpt;
    a.n_items = b->n_items;
    a.work = b->d_work;
    a.sc = b->sc;
    a.mode = b->es.mode;
    a.alpha = (float)b->es.alpha;
    a.q_total = (float)b->es.q_total;
    a.contract = b->contract;
    a.energy = energy;
    a.forces = forces;
    a.charges = charges;
    a.virial = virial;
    a.bec = out->bec;
    a.total_charge = out->total_charge;
    a.polarization = out->polarization;
    a.rot = b->d_rot;
    a.pos_in = positions;
    a.n_struct = n_struct;
    a.n_total = b->n_total;
    a.status = b->d_status;
    if (b->profiling) CKB(cudaEventRecord(b->ev[1], st));
    launch_batch_items(a, b->warps, b->nph_max, b->contract, std::min(slots, std::max(b->n_items, 1)), st);
    if (b->profiling) {
        CKB(cudaEventRecord(b->ev[2], st));
        b->pending = true;
    }
    CKB(cudaGetLastError());
    b->last_stream = st;
    return QNEP_OK;
}

qnep_status qnep_batch_sync_status(qnep_batch* b) {
    if (!b) return QNEP_ERR_ARG;
    CKB(cudaStreamSynchronize(b->last_stream));
    unsigned int w[2] = {0u, 0u};
    CKB(cudaMemcpy(w, b->d_status, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (w[1]) b->geom_valid = false;   // kept geometry with an error: the next call rebuilds it
    const qnep_status s = qnep_status_from_device_bits(w[0] | w[1]);
    if (s == QNEP_ERR_ARG) return failb(b, s, "a species index is outside [0, n_species)");
    if (s == QNEP_ERR_NBR_OVERFLOW) return failb(b, s, "neighbour list capacity exceeded");
    if (s == QNEP_ERR_TIMEOUT)
        return failb(b, s, "a bounded device-side wait gave up (a bulk copy or a tensor-core operation did not complete)");
    return QNEP_OK;
}

qnep_status qnep_batch_compute_host(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions_host,
                                    const int* types_host, const double* boxes, void* stream,
                                    const qnep_batch_outputs* out_host) {
    if (!b) return QNEP_ERR_ARG;
    if (n_struct < 1 || !atom_offsets || !boxes || !out_host || !out_host->energy)
        return failb(b, QNEP_ERR_ARG, "bad batch arguments");
    const int n_total = atom_offsets[n_struct];
    if (n_total < 0) return failb(b, QNEP_ERR_ARG, "atom_offsets must not decrease");
    if (n_total > 0 && (!positions_host || !types_host)) return failb(b, QNEP_ERR_ARG, "positions and types are required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t evals = (size_t)b->n_cand * (size_t)n_total, pairs = (size_t)b->n_cand * (size_t)n_struct;
    if ((size_t)n_total > b->io_atoms || evals > b->io_evals || pairs > b->io_pairs || !b->io_energy) {
        // device copies of the inputs and of every output, kept for the next call of this shape
        CKB(cudaStreamSynchronize(st));
        void* old[] = {b->io_pos, b->io_types, b->io_energy, b->io_forces, b->io_charges, b->io_virial, b->io_bec,
                       b->io_qtot, b->io_pol};
        for (void* q : old)
            if (q) cudaFree(q);
        b->io_pos = nullptr;
        b->io_types = nullptr;
        b->io_energy = nullptr;
        b->io_forces = nullptr;
        b->io_charges = nullptr;
        b->io_virial = nullptr;
        b->io_bec = nullptr;
        b->io_qtot = nullptr;
        b->io_pol = nullptr;
        b->io_atoms = b->io_evals = b->io_pairs = 0;
        const size_t na = std::max<size_t>(n_total, 1), ne = std::max<size_t>(evals, 1), np = std::max<size_t>(pairs, 1);
        CKB(cudaMalloc((void**)&b->io_pos, sizeof(float) * 3 * na));
        CKB(cudaMalloc((void**)&b->io_types, sizeof(int) * na));
        CKB(cudaMalloc((void**)&b->io_energy, sizeof(double) * np));
        CKB(cudaMalloc((void**)&b->io_forces, sizeof(float) * 3 * ne));
        CKB(cudaMalloc((void**)&b->io_charges, sizeof(float) * ne));
        CKB(cudaMalloc((void**)&b->io_virial, sizeof(double) * 9 * np));
        CKB(cudaMalloc((void**)&b->io_qtot, sizeof(double) * np));
        CKB(cudaMalloc((void**)&b->io_pol, sizeof(double) * 3 * np));
        b->io_atoms = na;
        b->io_evals = ne;
        b->io_pairs = np;
    }
    if (n_total > 0) {
        CKB(cudaMemcpyAsync(b->io_pos, positions_host, sizeof(float) * 3 * (size_t)n_total, cudaMemcpyHostToDevice, st));
        CKB(cudaMemcpyAsync(b->io_types, types_host, sizeof(int) * (size_t)n_total, cudaMemcpyHostToDevice, st));
    }
    if (out_host->bec && !b->io_bec) {   // BEC copies only for callers that ask for them (9 floats per evaluation)
        CKB(cudaStreamSynchronize(st));
        CKB(cudaMalloc((void**)&b->io_bec, sizeof(float) * 9 * b->io_evals));
    }
    qnep_batch_outputs dev{b->io_energy, out_host->forces ? b->io_forces : nullptr,
                           out_host->charges ? b->io_charges : nullptr, out_host->virial ? b->io_virial : nullptr,
                           out_host->bec ? b->io_bec : nullptr, out_host->total_charge ? b->io_qtot : nullptr,
                           out_host->polarization ? b->io_pol : nullptr};
    qnep_status s = qnep_batch_compute_outputs(b, n_struct, atom_offsets, b->io_pos, b->io_types, boxes, stream, &dev);
    if (s != QNEP_OK) return s;
    CKB(cudaMemcpyAsync(out_host->energy, b->io_energy, sizeof(double) * pairs, cudaMemcpyDeviceToHost, st));
    if (out_host->forces)
        CKB(cudaMemcpyAsync(out_host->forces, b->io_forces, sizeof(float) * 3 * evals, cudaMemcpyDeviceToHost, st));
    if (out_host->charges)
        CKB(cudaMemcpyAsync(out_host->charges, b->io_charges, sizeof(float) * evals, cudaMemcpyDeviceToHost, st));
    if (out_host->virial)
        CKB(cudaMemcpyAsync(out_host->virial, b->io_virial, sizeof(double) * 9 * pairs, cudaMemcpyDeviceToHost, st));
    if (out_host->bec)
        CKB(cudaMemcpyAsync(out_host->bec, b->io_bec, sizeof(float) * 9 * evals, cudaMemcpyDeviceToHost, st));
    if (out_host->total_charge)
        CKB(cudaMemcpyAsync(out_host->total_charge, b->io_qtot, sizeof(double) * pairs, cudaMemcpyDeviceToHost, st));
    if (out_host->polarization)
        CKB(cudaMemcpyAsync(out_host->polarization, b->io_pol, sizeof(double) * 3 * pairs, cudaMemcpyDeviceToHost, st));
    b->last_stream = st;
    return qnep_batch_sync_status(b);
}

qnep_status qnep_batch_debug_set_status(qnep_batch* b, unsigned int bits) {
    if (!b || !b->d_status) return QNEP_ERR_ARG;
    CKB(cudaDeviceSynchronize());
    unsigned int h = 0;
    CKB(cudaMemcpy(&h, b->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    h |= bits;
    CKB(cudaMemcpy(b->d_status, &h, sizeof(unsigned int), cudaMemcpyHostToDevice));
    return QNEP_OK;
}

qnep_status qnep_batch_autotune(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions,
                                const int* types, const double* boxes, void* stream, double* energy, float* forces,
                                float* charges, int reps, double* best_ms) {
    if (!b || reps < 1) return QNEP_ERR_ARG;
    std::vector<float> t;   // the event times of one shape's repetitions
    try {
        t.resize((size_t)reps);
    } catch (const std::bad_alloc&) {
        return failb(b, QNEP_ERR_OOM, "host memory for the autotuner's timings could not be obtained");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    const int shapes[2] = {8, 4};
    const int orders[2] = {QNEP_BATCH_ORDER_LARGEST_FIRST, QNEP_BATCH_ORDER_STRUCTURE};
    double best = 1e300;
    int bw = b->warps, bo = b->order_policy;
    qnep_status result = QNEP_OK;
    for (int w : shapes) {
        for (int o : orders) {
            b->warps = w;
            b->order_policy = o;
            qnep_status s = qnep_batch_compute(b, n_struct, atom_offsets, positions, types, boxes, stream, energy,
                                               forces, charges);
            if (s == QNEP_OK) s = qnep_batch_sync_status(b);
            if (s != QNEP_OK) {
                if (s == QNEP_ERR_UNSUPPORTED) continue;   // this block shape does not fit
                result = s;
                break;
            }
            for (int r = 0; r < reps && s == QNEP_OK; ++r) {
                cudaEventRecord(e0, st);
                s = qnep_batch_compute(b, n_struct, atom_offsets, positions, types, boxes, stream, energy, forces,
                                       charges);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&t[r], e0, e1);
            }
            if (s != QNEP_OK) {
                result = s;
                break;
            }
            std::sort(t.begin(), t.end());
            const double med = t[reps / 2];
            if (med < best) {
                best = med;
                bw = w;
                bo = o;
            }
        }
        if (result != QNEP_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->warps = bw;
    b->order_policy = bo;
    if (best_ms) *best_ms = best < 1e299 ? best : -1.0;
    return result;
}

qnep_status qnep_batch_set_profiling(qnep_batch* b, int enable) {
    if (!b) return QNEP_ERR_ARG;
    if (enable && !b->ev[0])
        for (auto& e : b->ev) CKB(cudaEventCreate(&e));
    b->profiling = enable != 0;
    b->pending = false;
    return QNEP_OK;
}

qnep_status qnep_batch_stage_times(qnep_batch* b, float* ms_out, int* n_calls) {
    if (!b || !ms_out || !n_calls) return QNEP_ERR_ARG;
    if (b->pending) {
        CKB(cudaEventSynchronize(b->ev[2]));
        float t0 = 0.f, t1 = 0.f;
        cudaEventElapsedTime(&t0, b->ev[0], b->ev[1]);
        cudaEventElapsedTime(&t1, b->ev[1], b->ev[2]);
        b->stage_ms[0] += t0;
        b->stage_ms[1] += t1;
        ++b->timed_calls;
        b->pending = false;
    }
    ms_out[0] = (float)b->stage_ms[0];
    ms_out[1] = (float)b->stage_ms[1];
    *n_calls = b->timed_calls;
    b->stage_ms[0] = b->stage_ms[1] = 0.0;
    b->timed_calls = 0;
    return QNEP_OK;
}

const char* qnep_batch_last_error(const qnep_batch* b) { return b ? b->err.c_str() : "null batch"; }

qnep_status qnep_batch_set_params(qnep_batch* b, const float* params, void* stream) {
    if (!b) return QNEP_ERR_ARG;
    if (!params) return failb(b, QNEP_ERR_ARG, "params is NULL");
    const int P = b->lay.total;
    dim3 grid((unsigned)((P + CG - 1) / CG), (unsigned)b->n_groups), block(CG, 8);
    k_set_params<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(params, b->d_pt, b->n_cand, P);
    CKB(cudaGetLastError());
    return QNEP_OK;
}

void qnep_batch_destroy(qnep_batch* b) {
    if (!b) return;
    if (b->last_stream) cudaStreamSynchronize(b->last_stream);
    void* ptrs[] = {b->d_pt,      b->d_st,     b->d_kt,       b->d_ktri,   b->d_rot,    b->d_chunk,  b->d_kvec,  b->d_kreal,     b->d_items_lpt,
                    b->d_items_nat, b->spos4,  b->sidx,       b->order,    b->spec_off,   b->cell_start,
                    b->nbr_list,  b->cnt_list, b->nbr_ang,    b->cnt_ang,  b->phase,      b->scratch,
                    b->geo_rad,   b->geo_ang,  b->bsum,     b->bimg,
                    b->d_work,    b->d_status, b->io_pos,   b->io_types, b->io_energy, b->io_forces,
                    b->io_charges, b->io_virial, b->io_bec, b->io_qtot, b->io_pol, b->zsum};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
