// Cell binning (atoms sorted by cell) and neighbour lists with periodic images.
//
// The paper evaluates every descriptor and real-space sum over neighbours
// within a cutoff (Sec. II.A radial / angular cutoffs; Sec. II.B real-space
// cutoff r_c); it does not describe the search.  Here:
//  * atoms are binned into cells no smaller than the list cutoff and reordered
//    by cell (then by input index, so the order is deterministic); every later
//    kernel works in this sorted order, outputs are scattered back at the end;
//  * per dimension the stencil reaches one cell to each side, each (cell, image
//    shift) visited once, so boxes with one or two cells per edge still see every
//    image within the cutoff (edge >= cutoff);
//  * one warp builds one atom's lists: the candidates of the 27 stencil cells are
//    flattened into one index space, 32 tested per step (one coalesced load each),
//    and a ballot compacts the accepted ones into shared memory; the lists are then
//    written grouped by neighbour species.
#include "nbr_common.cuh"

namespace qnep {

namespace {

// Wrap positions into the box, assign cells, count atoms per cell, clear the
// FP64 accumulators and (optionally) the structure-factor array of this call.
__global__ void k_bin(const float* __restrict__ pos, const int* __restrict__ types, int n, Geom g,
                      float4* __restrict__ pos4, int* __restrict__ cell_of, int* __restrict__ cell_count,
                      Accum* __restrict__ acc, double2* __restrict__ zero_buf, int zero_count,
                      const int* __restrict__ gate) {
    if (gate && *gate == 0) return;   // Verlet skin: the list is reused, positions come from k_skin_refresh
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        double* a = reinterpret_cast<double*>(acc);
        for (int k = 0; k < (int)(sizeof(Accum) / sizeof(double)); ++k) a[k] = 0.0;
    }
    for (int k = i; k < zero_count; k += gridDim.x * blockDim.x) zero_buf[k] = make_double2(0.0, 0.0);
    if (i >= n) return;
    float w[3];
    int cc[3];
    const float x[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    wrap_and_cell(g, x, w, cc);
    int t = types[i];
    pos4[i] = make_float4(w[0], w[1], w[2], __int_as_float(t));
    int c = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
}

// Exclusive scan of the cell counts (one block); clears the counts for the next call.
__global__ void k_scan(int* __restrict__ count, int ncells, int* __restrict__ start, int* __restrict__ fill,
                       const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ncells; base += blockDim.x) {
        int c = base + threadIdx.x;
        int v = c < ncells ? count[c] : 0;
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int nw = blockDim.x >> 5;
            int t = lane < nw ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) warp_tot[lane] = t;
        }
        __syncthreads();
        int excl = carry + x - v + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (c < ncells) {
            start[c] = excl;
            fill[c] = 0;
            count[c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncells] = carry;
}

__global__ void k_fill(const int* __restrict__ cell_of, int n, const int* __restrict__ start, int* __restrict__ fill,
                       int* __restrict__ slot_atoms, const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    int slot = atomicAdd(&fill[c], 1);
    slot_atoms[start[c] + slot] = i;
}

// One warp per cell: rank the cell's atoms by input index (the fill order is
// arbitrary) and write the sorted arrays: spos4[k], sidx[k] = input index.
__global__ void k_order(const int* __restrict__ start, int ncells, const int* __restrict__ slot_atoms,
                        const float4* __restrict__ pos4, float4* __restrict__ spos4, int* __restrict__ sidx, const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncells) return;
    const int s0 = start[c], cnt = start[c + 1] - s0;
    for (int a = lane; a - lane < cnt; a += 32) {
        int mine = a < cnt ? slot_atoms[s0 + a] : 0x7fffffff;
        int rank = 0;
        for (int b = 0; b < cnt; b += 32) {
            int other = (b + lane) < cnt ? slot_atoms[s0 + b + lane] : 0x7fffffff;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                int o = __shfl_sync(0xffffffffu, other, q);
                rank += (o < mine) ? 1 : 0;
            }
        }
        if (a < cnt) {
            spos4[s0 + rank] = pos4[mine];
            sidx[s0 + rank] = mine;
        }
    }
}

// Small systems (up to 2048 atoms): the four binning steps of k_bin, k_scan, k_fill and
// k_order in one block (counts, starts and fill cursors in shared memory), saving three
// launches and their latency.  Same outputs, same atom order (by cell, then by input
// index).  Measured: 192 atoms 17 -> 11 us for the binning; at 5000 atoms and more the
// single block is slower than the four grid-wide kernels.
constexpr int SMALL_BIN_ATOMS = 2048, SMALL_BIN_CELLS = 4096, SMALL_BIN_THREADS = 1024;

__global__ void __launch_bounds__(SMALL_BIN_THREADS) k_bin_small(const float* __restrict__ pos,
                                                                  const int* __restrict__ types, int n, Geom g,
                                                                  float4* __restrict__ pos4, int* __restrict__ cell_of,
                                                                  int* __restrict__ cell_start,
                                                                  int* __restrict__ slot_atoms,
                                                                  float4* __restrict__ spos4, int* __restrict__ sidx,
                                                                  Accum* __restrict__ acc,
                                                                  double2* __restrict__ zero_buf, int zero_count, const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ int cnt[SMALL_BIN_CELLS];
    __shared__ int start[SMALL_BIN_CELLS + 1];
    __shared__ int warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
    const int ncells = g.ncells;
    if (tid == 0) {
        double* a = reinterpret_cast<double*>(acc);
        for (int k = 0; k < (int)(sizeof(Accum) / sizeof(double)); ++k) a[k] = 0.0;
    }
    for (int k = tid; k < zero_count; k += nt) zero_buf[k] = make_double2(0.0, 0.0);
    for (int c = tid; c < ncells; c += nt) cnt[c] = 0;
    __syncthreads();
    // wrap, cell of each atom, counts
    for (int i = tid; i < n; i += nt) {
        float w[3];
        int cc[3];
        const float x[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        wrap_and_cell(g, x, w, cc);
        pos4[i] = make_float4(w[0], w[1], w[2], __int_as_float(types[i]));
        const int c = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
        cell_of[i] = c;
        atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    // exclusive scan of the counts (chunks of nt cells, carried)
    int carry = 0;
    for (int base = 0; base < ncells; base += nt) {
        const int c = base + tid;
        const int v = c < ncells ? cnt[c] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const int nw = nt >> 5;
            int t = lane < nw ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;   // inclusive warp prefix; lane 31 holds the chunk total
        }
        __syncthreads();
        const int excl = carry + x - v + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (c < ncells) start[c] = excl;
        carry += warp_tot[31];
        __syncthreads();   // warp_tot is rewritten by the next chunk
    }
    if (tid == 0) start[ncells] = carry;
    for (int c = tid; c < ncells; c += nt) cnt[c] = 0;   // fill cursors
    __syncthreads();
    for (int c = tid; c <= ncells; c += nt) cell_start[c] = start[c];
    for (int i = tid; i < n; i += nt) {
        const int c = cell_of[i];
        slot_atoms[start[c] + atomicAdd(&cnt[c], 1)] = i;
    }
    __syncthreads();
    // one warp per cell: rank the cell's atoms by input index
    for (int c = wid; c < ncells; c += nt >> 5) {
        const int s0 = start[c], m = start[c + 1] - s0;
        for (int a = lane; a - lane < m; a += 32) {
            const int mine = a < m ? slot_atoms[s0 + a] : 0x7fffffff;
            int rank = 0;
            for (int b = 0; b < m; b += 32) {
                const int other = (b + lane) < m ? slot_atoms[s0 + b + lane] : 0x7fffffff;
#pragma unroll 8
                for (int q = 0; q < 32; ++q) rank += (__shfl_sync(0xffffffffu, other, q) < mine) ? 1 : 0;
            }
            if (a < m) {
                spos4[s0 + rank] = pos4[mine];
                sidx[s0 + rank] = mine;
            }
        }
    }
}

__global__ void k_neighbors(const float4* __restrict__ spos4, const int* __restrict__ cell_start, int n,
                            int n_species, Geom g, int cap_list, int cap_ang, int* __restrict__ nbr_list,
                            int* __restrict__ cnt_list, int* __restrict__ nbr_ang, int* __restrict__ cnt_ang,
                            Accum* __restrict__ acc) {
    extern __shared__ int nsm[];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int* sl = nsm + wib * (cap_list + cap_ang) * 2;
    int* slt = sl + cap_list;
    int* sa = slt + cap_list;
    int* sat = sa + cap_ang;
    if (k >= n) return;
    const float4 pk = spos4[k];
    int nl = 0, na = 0;
    bool ovf = warp_build_lists(spos4, cell_start, k, pk, g, cap_list, cap_ang, sl, slt, sa, sat, nl, na);
    warp_write_grouped(sl, slt, nl, n_species, n, k, nbr_list, (size_t)g.list_sa, (size_t)g.list_se, cnt_list);
    warp_write_grouped(sa, sat, na, n_species, n, k, nbr_ang, (size_t)g.ang_sa, (size_t)g.ang_se, cnt_ang);
    if (ovf && lane == 0) atomicOr(&acc->status, 1u);
}

}  // namespace

void launch_bin(const float* pos, const int* types, int n, const Geom& g, float4* pos4, int* cell_of, int* cell_count,
                int* cell_start, int* cell_fill, int* slot_atoms, float4* spos4, int* sidx, Accum* acc,
                double2* zero_buf, int zero_count, cudaStream_t st, const int* gate) {
    if (n <= SMALL_BIN_ATOMS && g.ncells <= SMALL_BIN_CELLS && zero_count <= 64 * SMALL_BIN_THREADS) {
        // counts in shared memory: cell_count / cell_fill are not used (and stay zero)
        k_bin_small<<<1, SMALL_BIN_THREADS, 0, st>>>(pos, types, n, g, pos4, cell_of, cell_start, slot_atoms, spos4,
                                                     sidx, acc, zero_buf, zero_count, gate);
        return;
    }
    int blocks = (n + 255) / 256;
    int zb = (zero_count + 255) / 256;
    if (zb > blocks) blocks = zb;
    if (blocks < 1) blocks = 1;
    k_bin<<<blocks, 256, 0, st>>>(pos, types, n, g, pos4, cell_of, cell_count, acc, zero_buf, zero_count, gate);
    k_scan<<<1, 1024, 0, st>>>(cell_count, g.ncells, cell_start, cell_fill, gate);
    if (n > 0) {
        k_fill<<<(n + 255) / 256, 256, 0, st>>>(cell_of, n, cell_start, cell_fill, slot_atoms, gate);
        k_order<<<(g.ncells * 32 + 127) / 128, 128, 0, st>>>(cell_start, g.ncells, slot_atoms, pos4, spos4, sidx,
                                                              gate);
    }
}

// ---- Verlet skin ----------------------------------------------------------------------------
// A candidate list with cutoff r_list + skin is kept while no atom has moved more than skin / 2
// since it was built: then every pair now within r_list was within r_list + skin at the build,
// so filtering the candidates by the current distances gives exactly the lists of a fresh cell
// search (in another order).  The test and the choice between rebuilding and reusing are made
// on the device (a gate word), so a step needs no host synchronisation:
//   k_skin_check    gate = 1 if |x_i - x_i^ref| > skin / 2 for any atom (the host sets the gate
//                   to 1 instead when there is no valid list: first call, new box or size)
//   gate = 1:       the binning kernels sort the atoms again, k_skin_build writes the candidate
//                   lists, the reference positions (input order) and the sorted positions at the build
//   gate = 0:       k_skin_refresh moves the sorted positions by the displacement since the build
//                   (not wrapped into the box: the stored image shifts stay valid) and clears the
//                   accumulators as the binning would
__global__ void k_skin_check(const float* __restrict__ pos, const float* __restrict__ xref, int n, float lim2,
                             int* __restrict__ gate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dx = pos[3 * i] - xref[3 * i], dy = pos[3 * i + 1] - xref[3 * i + 1], dz = pos[3 * i + 2] - xref[3 * i + 2];
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (!(d2 <= lim2)) *gate = 1;   // also a non-finite displacement
}

__global__ void __launch_bounds__(128) k_skin_build(const float4* __restrict__ spos4, const int* __restrict__ cell_start,
                                                    const int* __restrict__ sidx, const float* __restrict__ pos, int n,
                                                    Geom gs, int cap_s, int* __restrict__ skin_list,
                                                    int* __restrict__ skin_cnt, float4* __restrict__ sref4,
                                                    float* __restrict__ xref, const int* __restrict__ gate,
                                                    Accum* __restrict__ acc, unsigned int* __restrict__ rebuilds) {
    if (*gate == 0) return;
    extern __shared__ int ksm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(rebuilds, 1u);
    if (k >= n) return;
    int* sl = ksm + wib * 2 * cap_s;
    int* slt = sl + cap_s;
    const float4 pk = spos4[k];
    int nl = 0, na = 0;
    // gs: list cutoff r_list + skin, no angular part (rc_angular 0, capacity 0)
    const bool ovf = warp_build_lists(spos4, cell_start, k, pk, gs, cap_s, 0, sl, slt, nullptr, nullptr, nl, na);
    for (int e = lane; e < nl; e += 32) skin_list[(size_t)k * cap_s + e] = sl[e];
    if (lane == 0) {
        skin_cnt[k] = nl;
        sref4[k] = pk;
        const int i = sidx[k];
        xref[3 * i] = pos[3 * i];
        xref[3 * i + 1] = pos[3 * i + 1];
        xref[3 * i + 2] = pos[3 * i + 2];
        if (ovf) atomicOr(&acc->status, 1u);
    }
}

__global__ void k_skin_refresh(const float* __restrict__ pos, const float* __restrict__ xref,
                               const float4* __restrict__ sref4, const int* __restrict__ sidx, int n,
                               const int* __restrict__ gate, Accum* __restrict__ acc, double2* __restrict__ zero_buf,
                               int zero_count, float4* __restrict__ spos4) {
    if (*gate != 0) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        double* a = reinterpret_cast<double*>(acc);
        for (int q = 0; q < (int)(sizeof(Accum) / sizeof(double)); ++q) a[q] = 0.0;
    }
    for (int q = t; q < zero_count; q += gridDim.x * blockDim.x) zero_buf[q] = make_double2(0.0, 0.0);
    if (t >= n) return;
    const int i = sidx[t];
    const float4 r = sref4[t];
    spos4[t] = make_float4(r.x + (pos[3 * i] - xref[3 * i]), r.y + (pos[3 * i + 1] - xref[3 * i + 1]),
                           r.z + (pos[3 * i + 2] - xref[3 * i + 2]), r.w);
}

void launch_skin(const float* pos, const int* types, int n, const Geom& g, float skin, bool force, int cap_s,
                 float4* pos4, int* cell_of, int* cell_count, int* cell_start, int* cell_fill, int* slot_atoms,
                 float4* spos4, int* sidx, Accum* acc, double2* zero_buf, int zero_count, int* gate, int* skin_list,
                 int* skin_cnt, float4* sref4, float* xref, unsigned int* rebuilds, cudaStream_t st) {
    // the gate is read as zero / non-zero: without a valid list it starts non-zero (every byte 1)
    cudaMemsetAsync(gate, force ? 1 : 0, sizeof(int), st);
    if (!force) {
        const float h = 0.5f * skin;
        k_skin_check<<<(n + 255) / 256, 256, 0, st>>>(pos, xref, n, h * h, gate);
    }
    launch_bin(pos, types, n, g, pos4, cell_of, cell_count, cell_start, cell_fill, slot_atoms, spos4, sidx, acc,
               zero_buf, zero_count, st, gate);
    Geom gs = g;
    gs.rc_list = g.rc_list + skin;
    gs.rc_angular = 0.f;
    const size_t smem = sizeof(int) * 4 * 2 * (size_t)cap_s;
    static std::atomic<int> attr[kMaxDevices];
    if (smem > 48 * 1024) ensure_smem_attr(k_skin_build, attr, (int)smem);
    k_skin_build<<<(n + 3) / 4, 128, smem, st>>>(spos4, cell_start, sidx, pos, n, gs, cap_s, skin_list, skin_cnt,
                                                 sref4, xref, gate, acc, rebuilds);
    const int zb = std::max((n + 255) / 256, (zero_count + 255) / 256);
    k_skin_refresh<<<std::max(zb, 1), 256, 0, st>>>(pos, xref, sref4, sidx, n, gate, acc, zero_buf, zero_count, spos4);
}

void launch_neighbors(const float4* spos4, const int* cell_start, int n, int n_species, const Geom& g, int cap_list,
                      int cap_ang, int* nbr_list, int* cnt_list, int* nbr_ang, int* cnt_ang, Accum* acc,
                      cudaStream_t st) {
    if (n == 0) return;
    const int threads = 128;
    size_t smem = sizeof(int) * (threads / 32) * (cap_list + cap_ang) * 2;
    static std::atomic<int> attr[kMaxDevices];
    ensure_smem_attr(k_neighbors, attr, 200 * 1024);
    long long blocks = ((long long)n * 32 + threads - 1) / threads;
    k_neighbors<<<(unsigned)blocks, threads, smem, st>>>(spos4, cell_start, n, n_species, g, cap_list, cap_ang,
                                                        nbr_list, cnt_list, nbr_ang, cnt_ang, acc);
}

}  // namespace qnep
