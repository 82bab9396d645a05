// Cell binning and neighbour lists (periodic images included).
//
// The paper evaluates every descriptor and real-space sum over neighbours
// within a cutoff (Sec. II.A radial / angular cutoffs; Sec. II.B real-space
// cutoff r_c); it does not describe the search.  Here: a cell grid with cells
// no smaller than the list cutoff; per dimension the stencil reaches one cell
// to each side, each (cell, image shift) visited once, so boxes with only one
// or two cells per edge still see every image within the cutoff (edge >= cutoff).
// One warp builds the lists of one atom: lanes test 32 candidates at a time
// and a ballot compacts the accepted ones in a fixed order (neighbour species,
// stencil cell, atom index) so that lists are deterministic.
#include "qnep_internal.cuh"

namespace qnep {

namespace {

__device__ __forceinline__ int cell_coord(float x, float invL, int nc) {
    int c = (int)(x * invL * (float)nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_bin(const float* __restrict__ pos, const int* __restrict__ types, int n, Geom g,
                      float4* __restrict__ pos4, int* __restrict__ cell_of, int* __restrict__ cell_count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float w[3];
    for (int d = 0; d < 3; ++d) {
        float x = pos[3 * i + d];
        float f = floorf(x * g.invL[d]);
        float y = fmaf(-f, g.L[d], x);
        if (y >= g.L[d]) y -= g.L[d];
        if (y < 0.f) y += g.L[d];
        if (y >= g.L[d]) y = 0.f;
        w[d] = y;
    }
    int t = types[i];
    pos4[i] = make_float4(w[0], w[1], w[2], __int_as_float(t));
    int c = (cell_coord(w[2], g.invL[2], g.nc[2]) * g.nc[1] + cell_coord(w[1], g.invL[1], g.nc[1])) * g.nc[0] +
            cell_coord(w[0], g.invL[0], g.nc[0]);
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
}

// Exclusive scan of the cell counts (one block, any number of cells).
__global__ void k_scan(const int* __restrict__ count, int ncells, int* __restrict__ start,
                       int* __restrict__ fill) {
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
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncells] = carry;
}

__global__ void k_fill(const int* __restrict__ cell_of, int n, const int* __restrict__ start,
                       int* __restrict__ fill, int* __restrict__ atoms) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    int slot = atomicAdd(&fill[c], 1);
    atoms[start[c] + slot] = i;
}

// Sort each cell's atoms by (species, index): deterministic lists grouped by species.
__global__ void k_sort_cells(const int* __restrict__ start, int ncells, const float4* __restrict__ pos4,
                             int* __restrict__ atoms) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int s0 = start[c], s1 = start[c + 1];
    for (int a = s0 + 1; a < s1; ++a) {
        int v = atoms[a];
        long long key = ((long long)__float_as_int(pos4[v].w) << 32) | (unsigned)v;
        int b = a - 1;
        while (b >= s0) {
            int u = atoms[b];
            long long ku = ((long long)__float_as_int(pos4[u].w) << 32) | (unsigned)u;
            if (ku <= key) break;
            atoms[b + 1] = u;
            --b;
        }
        atoms[b + 1] = v;
    }
}

__global__ void k_neighbors(const float4* __restrict__ pos4, const int* __restrict__ cell_start,
                            const int* __restrict__ cell_atoms, int n, int n_species, Geom g, int cap_list,
                            int cap_ang, int* __restrict__ nbr_list, int* __restrict__ cnt_list,
                            int* __restrict__ nbr_ang, int* __restrict__ cnt_ang, Accum* __restrict__ acc) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp;
    const float4 pi = pos4[i];
    int ci[3];
    ci[0] = cell_coord(pi.x, g.invL[0], g.nc[0]);
    ci[1] = cell_coord(pi.y, g.invL[1], g.nc[1]);
    ci[2] = cell_coord(pi.z, g.invL[2], g.nc[2]);
    const float rl2 = g.rc_list * g.rc_list;
    const float ra2 = g.rc_angular * g.rc_angular;
    int nl = 0, na = 0;
    bool overflow = false;
    for (int s = 0; s < n_species; ++s) {
        int nl0 = nl, na0 = na;
        for (int dz = -1; dz <= 1; ++dz) {
            int cz = ci[2] + dz;
            int tz = cz < 0 ? -1 : (cz >= g.nc[2] ? 1 : 0);
            cz -= tz * g.nc[2];
            for (int dy = -1; dy <= 1; ++dy) {
                int cy = ci[1] + dy;
                int ty = cy < 0 ? -1 : (cy >= g.nc[1] ? 1 : 0);
                cy -= ty * g.nc[1];
                for (int dx = -1; dx <= 1; ++dx) {
                    int cx = ci[0] + dx;
                    int tx = cx < 0 ? -1 : (cx >= g.nc[0] ? 1 : 0);
                    cx -= tx * g.nc[0];
                    int c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
                    int code = (tx + 1) + 3 * (ty + 1) + 9 * (tz + 1);
                    float sx = tx * g.L[0] - pi.x, sy = ty * g.L[1] - pi.y, sz = tz * g.L[2] - pi.z;
                    int b0 = cell_start[c], b1 = cell_start[c + 1];
                    for (int b = b0; b < b1; b += 32) {
                        int k = b + lane;
                        bool inl = false, ina = false;
                        int j = 0;
                        if (k < b1) {
                            j = cell_atoms[k];
                            float4 pj = pos4[j];
                            if (__float_as_int(pj.w) == s && !(j == i && code == 13)) {
                                float vx = pj.x + sx, vy = pj.y + sy, vz = pj.z + sz;
                                float r2 = vx * vx + vy * vy + vz * vz;
                                inl = r2 < rl2;
                                ina = r2 < ra2;
                            }
                        }
                        unsigned ml = __ballot_sync(0xffffffffu, inl);
                        unsigned ma = __ballot_sync(0xffffffffu, ina);
                        unsigned below = (1u << lane) - 1u;
                        int e = j | (code << CODE_SHIFT);
                        if (inl) {
                            int slot = nl + __popc(ml & below);
                            if (slot < cap_list) nbr_list[(size_t)slot * n + i] = e;
                        }
                        if (ina) {
                            int slot = na + __popc(ma & below);
                            if (slot < cap_ang) nbr_ang[(size_t)slot * n + i] = e;
                        }
                        nl += __popc(ml);
                        na += __popc(ma);
                    }
                }
            }
        }
        if (nl > cap_list || na > cap_ang) overflow = true;
        int cl = min(nl, cap_list) - min(nl0, cap_list);
        int ca = min(na, cap_ang) - min(na0, cap_ang);
        if (lane == 0) {
            cnt_list[(size_t)s * n + i] = cl;
            cnt_ang[(size_t)s * n + i] = ca;
        }
    }
    if (overflow && lane == 0) atomicOr(&acc->status, 1u);
}

}  // namespace

void launch_bin(const float* pos, const int* types, int n, const Geom& g, float4* pos4, int* cell_of,
                int* cell_count, int* cell_start, int* cell_fill, int* cell_atoms, cudaStream_t st) {
    cudaMemsetAsync(cell_count, 0, sizeof(int) * g.ncells, st);
    if (n > 0) k_bin<<<(n + 255) / 256, 256, 0, st>>>(pos, types, n, g, pos4, cell_of, cell_count);
    k_scan<<<1, 1024, 0, st>>>(cell_count, g.ncells, cell_start, cell_fill);
    if (n > 0) {
        k_fill<<<(n + 255) / 256, 256, 0, st>>>(cell_of, n, cell_start, cell_fill, cell_atoms);
        k_sort_cells<<<(g.ncells + 127) / 128, 128, 0, st>>>(cell_start, g.ncells, pos4, cell_atoms);
    }
}

void launch_neighbors(const float4* pos4, const int* cell_start, const int* cell_atoms, int n,
                      int n_species, const Geom& g, int cap_list, int cap_ang, int* nbr_list,
                      int* cnt_list, int* nbr_ang, int* cnt_ang, Accum* acc, cudaStream_t st) {
    if (n == 0) return;
    const int threads = 128;
    long long blocks = ((long long)n * 32 + threads - 1) / threads;
    k_neighbors<<<(unsigned)blocks, threads, 0, st>>>(pos4, cell_start, cell_atoms, n, n_species, g, cap_list,
                                                      cap_ang, nbr_list, cnt_list, nbr_ang, cnt_ang, acc);
}

}  // namespace qnep
