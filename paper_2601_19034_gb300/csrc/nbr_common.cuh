// Warp-level neighbour-list construction shared by the list kernel and the
// fused neighbour + descriptor kernel.
#pragma once

#include "qnep_internal.cuh"

namespace qnep {

__device__ __forceinline__ int nbr_cell_coord(float x, float invL, int nc) {
    int c = (int)(x * invL * (float)nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Build the lists of sorted atom k (position pk) into shared memory.
//   sl / slt: list entries (index | image code << 26) and neighbour species, capacity cap_l
//   sa / sat: angular entries and species, capacity cap_a
// The candidates of the 27 stencil cells (visited in order, atoms in cell order) form one
// index space scanned 4 x 32 at a time: lane t finds its cell by a binary search over the
// cells' prefix counts (shuffles), tests its candidate, and a ballot compacts the accepted
// ones.  nl / na return the number of entries stored (clamped to the capacities); the return
// value is true when a capacity was exceeded.  Whole warp only.
__device__ __forceinline__ bool warp_build_lists(const float4* __restrict__ spos4, const int* __restrict__ cell_start,
                                                 int k, float4 pk, const Geom& g, int cap_l, int cap_a, int* sl,
                                                 int* slt, int* sa, int* sat, int& nl, int& na) {
    const int lane = threadIdx.x & 31;
    // lane s < 27 describes stencil cell s: first atom, atom count, image shift code and vector
    int cstart = 0, ccnt = 0, code = CODE_SELF;
    float tx = 0.f, ty = 0.f, tz = 0.f;
    if (lane < 27) {
        int d[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        // the atom's cell: from the position (orthorhombic) or its fractional coordinates
        float p[3] = {pk.x, pk.y, pk.z};
        if (g.tri) {
            float sf[3];
            frac_of(g, pk.x, pk.y, pk.z, sf);
            for (int q = 0; q < 3; ++q) p[q] = sf[q];
        }
        int cc[3], tt[3];
        for (int q = 0; q < 3; ++q) {
            int c = (g.tri ? nbr_cell_coord(p[q], 1.f, g.nc[q]) : nbr_cell_coord(p[q], g.invL[q], g.nc[q])) + d[q];
            int t = c < 0 ? -1 : (c >= g.nc[q] ? 1 : 0);
            cc[q] = c - t * g.nc[q];
            tt[q] = t;
        }
        int c = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
        cstart = cell_start[c];
        ccnt = cell_start[c + 1] - cstart;
        code = (tt[0] + 1) | ((tt[1] + 1) << 2) | ((tt[2] + 1) << 4);
        shift_vector(g, (float)tt[0], (float)tt[1], (float)tt[2], tx, ty, tz);
    }
    // inclusive prefix counts over the 27 cells (lanes 27..31 add nothing)
    int incl = ccnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - ccnt;
    const float rl2 = g.rc_list * g.rc_list;
    const float ra2 = g.rc_angular * g.rc_angular;
    const unsigned below = (1u << lane) - 1u;
    int cl = 0, ca = 0;
    // four rounds of 32 candidates per iteration: the four position loads are in flight together
    for (int base = 0; base < total; base += 128) {
        int mm[4], cdd[4];
        float sxx[4], syy[4], szz[4];
        float4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = base + 32 * u + lane;
            // cell of candidate t: the last cell s with excl[s] <= t (binary search over lanes 0..26)
            int s = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int probe = s + step;
                const int ex = __shfl_sync(0xffffffffu, excl, probe < 27 ? probe : 26);
                if (probe < 27 && ex <= t) s = probe;
            }
            const int c0 = __shfl_sync(0xffffffffu, cstart, s);
            const int e0 = __shfl_sync(0xffffffffu, excl, s);
            cdd[u] = __shfl_sync(0xffffffffu, code, s);
            sxx[u] = __shfl_sync(0xffffffffu, tx, s);
            syy[u] = __shfl_sync(0xffffffffu, ty, s);
            szz[u] = __shfl_sync(0xffffffffu, tz, s);
            mm[u] = c0 + (t - e0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            pj[u] = base + 32 * u + lane < total ? __ldg(&spos4[mm[u]]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (base + 32 * u >= total) break;   // warp-uniform
            const int t = base + 32 * u + lane;
            const int m = mm[u], cd = cdd[u];
            bool inl = false, ina = false;
            int typ = 0;
            if (t < total) {
                float vx = (pj[u].x - pk.x) + sxx[u], vy = (pj[u].y - pk.y) + syy[u], vz = (pj[u].z - pk.z) + szz[u];
                float r2 = vx * vx + vy * vy + vz * vz;
                inl = r2 < rl2 && !(m == k && cd == CODE_SELF);
                ina = inl && r2 < ra2;
                typ = __float_as_int(pj[u].w);
            }
            const unsigned ml = __ballot_sync(0xffffffffu, inl);
            const unsigned ma = __ballot_sync(0xffffffffu, ina);
            const int ent = (int)((unsigned)m | ((unsigned)cd << CODE_SHIFT));
            if (inl) {
                int slot = cl + __popc(ml & below);
                if (slot < cap_l) {
                    sl[slot] = ent;
                    slt[slot] = typ;
                }
            }
            if (ina) {
                int slot = ca + __popc(ma & below);
                if (slot < cap_a) {
                    sa[slot] = ent;
                    sat[slot] = typ;
                }
            }
            cl += __popc(ml);
            ca += __popc(ma);
        }
    }
    __syncwarp();
    nl = cl < cap_l ? cl : cap_l;
    na = ca < cap_a ? ca : cap_a;
    return cl > cap_l || ca > cap_a;
}

// The lists of sorted atom k from its Verlet-skin candidates cand[0..total) (entries with image
// codes, built with a longer cutoff): the same tests, staging and return value as
// warp_build_lists, on the current positions.  Whole warp only.
__device__ __forceinline__ bool warp_lists_from_skin(const float4* __restrict__ spos4, const int* __restrict__ cand,
                                                     int total, float4 pk, const Geom& g, int cap_l, int cap_a,
                                                     int* sl, int* slt, int* sa, int* sat, int& nl, int& na) {
    const int lane = threadIdx.x & 31;
    const float rl2 = g.rc_list * g.rc_list;
    const float ra2 = g.rc_angular * g.rc_angular;
    const unsigned below = (1u << lane) - 1u;
    int cl = 0, ca = 0;
    for (int base = 0; base < total; base += 128) {
        int ent[4];
        float4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = base + 32 * u + lane;
            ent[u] = t < total ? __ldg(&cand[t]) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            pj[u] = base + 32 * u + lane < total ? __ldg(&spos4[ent[u] & INDEX_MASK]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (base + 32 * u >= total) break;   // warp-uniform
            const int t = base + 32 * u + lane;
            bool inl = false, ina = false;
            int typ = 0;
            if (t < total) {
                const unsigned code = (unsigned)ent[u] >> CODE_SHIFT;
                float sx, sy, sz;
                shift_vector(g, (float)((int)(code & 3u) - 1), (float)((int)((code >> 2) & 3u) - 1),
                             (float)((int)(code >> 4) - 1), sx, sy, sz);
                const float vx = (pj[u].x - pk.x) + sx, vy = (pj[u].y - pk.y) + sy, vz = (pj[u].z - pk.z) + sz;
                const float r2 = vx * vx + vy * vy + vz * vz;
                inl = r2 < rl2;
                ina = inl && r2 < ra2;
                typ = __float_as_int(pj[u].w);
            }
            const unsigned ml = __ballot_sync(0xffffffffu, inl);
            const unsigned ma = __ballot_sync(0xffffffffu, ina);
            if (inl) {
                const int slot = cl + __popc(ml & below);
                if (slot < cap_l) {
                    sl[slot] = ent[u];
                    slt[slot] = typ;
                }
            }
            if (ina) {
                const int slot = ca + __popc(ma & below);
                if (slot < cap_a) {
                    sa[slot] = ent[u];
                    sat[slot] = typ;
                }
            }
            cl += __popc(ml);
            ca += __popc(ma);
        }
    }
    __syncwarp();
    nl = cl < cap_l ? cl : cap_l;
    na = ca < cap_a ? ca : cap_a;
    return cl > cap_l || ca > cap_a;
}

// Write staged entries grouped by neighbour species: out[k * sa + slot * se], counts cnt[s][n].
__device__ __forceinline__ void warp_write_grouped(const int* se_buf, const int* st_buf, int cnt, int n_species, int n,
                                                   int k, int* __restrict__ out, size_t stride_atom,
                                                   size_t stride_entry, int* __restrict__ out_cnt) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int off = 0;
    for (int s = 0; s < n_species; ++s) {
        const int c0 = off;
        for (int base = 0; base < cnt; base += 32) {
            const int e = base + lane;
            const bool take = e < cnt && st_buf[e] == s;
            const unsigned mk = __ballot_sync(0xffffffffu, take);
            if (take) out[(size_t)k * stride_atom + (size_t)(off + __popc(mk & below)) * stride_entry] = se_buf[e];
            off += __popc(mk);
        }
        if (lane == 0) out_cnt[(size_t)s * n + k] = off - c0;
    }
}

}  // namespace qnep
