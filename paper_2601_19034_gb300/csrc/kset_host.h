// Host construction of the half-space Ewald k-set (shared by the single-structure
// and the batched force calls).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

namespace qnep {

// Wave vectors k = 2 pi (n1/Lx, n2/Ly, n3/Lz) with 0 < |k| < kmax in the half space
// n1 > 0, or n1 = 0 and n2 > 0, or n1 = n2 = 0 and n3 > 0 (S(-k) = S(k)^*).  They
// are grouped in columns (n1, n2) holding the contiguous run n3 in [lo, hi], and each
// column is stored as 8-wide chunks of n3, padded past hi with G = 0.
struct KSet {
    int nmax[3];
    std::vector<int4> cols;       // (n1, n2, lo, padded offset); last entry (0, 0, 0, nk)
    std::vector<int> chunk_col;   // column of each chunk
    std::vector<float> kg;        // G(k) = (2 pi / V) exp(-k^2 / 4 alpha^2) / k^2, 0 on padding
};

// A general cell (rows a, b, c) turned into the restricted form a' = (a_x, 0, 0),
// b' = (b_x, b_y, 0), c' = (c_x, c_y, c_z): R has the rows e1 = a / |a|, e2 = e3 x e1,
// e3 = a x b / |a x b| (a rotation: orthonormal rows, det +1), and the rows of the turned cell
// are R a, R b, R c, with the entries zero by construction set to zero.  Returns false for a
// degenerate cell (a = 0 or a parallel to b); a left-handed cell comes out with c'_z < 0.
inline bool rotate_to_restricted(const double box[9], double R[9], double out[9]) {
    const double* av = box;
    const double* bv = box + 3;
    const double la = std::sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
    const double n3[3] = {av[1] * bv[2] - av[2] * bv[1], av[2] * bv[0] - av[0] * bv[2], av[0] * bv[1] - av[1] * bv[0]};
    const double ln = std::sqrt(n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2]);
    if (!(la > 0) || !(ln > 0)) return false;
    for (int d = 0; d < 3; ++d) {
        R[d] = av[d] / la;
        R[6 + d] = n3[d] / ln;
    }
    R[3] = R[7] * R[2] - R[8] * R[1];   // e2 = e3 x e1
    R[4] = R[8] * R[0] - R[6] * R[2];
    R[5] = R[6] * R[1] - R[7] * R[0];
    for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d)
            out[3 * r + d] = R[3 * d] * box[3 * r] + R[3 * d + 1] * box[3 * r + 1] + R[3 * d + 2] * box[3 * r + 2];
    out[1] = out[2] = out[5] = 0.0;
    return true;
}

// Phase factors per atom of the k-set whose axes have the lengths len[3] (the edges of an
// orthorhombic cell, the row lengths |a_d| of a general one): (n1max + 1) + (2 n2max + 1) +
// (2 n3max + 8), with n_d max = floor(k_max len_d / 2 pi) formed as the builders below form it, but
// in double and before any enumeration, so that a huge k_max * length is refused without an int
// overflow or a long host loop.  +inf when a product is not finite.
inline double kset_phase_count(const double len[3], double kmax) {
    const double two_pi = 6.283185307179586;
    double nm[3];
    for (int d = 0; d < 3; ++d) {
        nm[d] = std::floor(kmax * len[d] / two_pi);
        if (!std::isfinite(nm[d])) return HUGE_VAL;
    }
    return (nm[0] + 1) + (2 * nm[1] + 1) + (2 * nm[2] + 8);
}

inline KSet build_kset(const double L[3], double kmax, double alpha) {
    const double two_pi = 6.283185307179586;
    const double vol = L[0] * L[1] * L[2];
    KSet ks;
    for (int d = 0; d < 3; ++d) ks.nmax[d] = (int)std::floor(kmax * L[d] / two_pi);
    const int* nmax = ks.nmax;
    for (int n1 = 0; n1 <= nmax[0]; ++n1) {
        for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2) {
            if (n1 == 0 && n2 < 0) continue;
            double kx = two_pi * n1 / L[0], ky = two_pi * n2 / L[1];
            int lo = 1 << 30, hi = -(1 << 30);
            for (int n3 = -nmax[2]; n3 <= nmax[2]; ++n3) {
                if (n1 == 0 && n2 == 0 && n3 <= 0) continue;
                double kz = two_pi * n3 / L[2];
                double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > 0 && k2 < kmax * kmax) {
                    lo = std::min(lo, n3);
                    hi = std::max(hi, n3);
                }
            }
            if (hi < lo) continue;
            int nchunk = (hi - lo + 1 + 7) / 8;
            int c = (int)ks.cols.size();
            ks.cols.push_back(make_int4(n1, n2, lo, (int)ks.kg.size()));
            for (int h = 0; h < nchunk; ++h) ks.chunk_col.push_back(c);
            for (int t = 0; t < 8 * nchunk; ++t) {
                int n3 = lo + t;
                double kz = two_pi * n3 / L[2];
                double k2 = kx * kx + ky * ky + kz * kz;
                bool ok = n3 <= hi && k2 > 0 && k2 < kmax * kmax && !(n1 == 0 && n2 == 0 && n3 <= 0);
                ks.kg.push_back(ok ? (float)(two_pi / vol * std::exp(-k2 / (4 * alpha * alpha)) / k2) : 0.f);
            }
        }
    }
    ks.cols.push_back(make_int4(0, 0, 0, (int)ks.kg.size()));
    return ks;
}

// Inverse of a 3 x 3 row-major matrix; returns the determinant (0: singular, inverse not written).
inline double invert3(const double h[9], double hi[9]) {
    const double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                       h[2] * (h[3] * h[7] - h[4] * h[6]);
    if (det == 0.0) return 0.0;
    const double id = 1.0 / det;
    hi[0] = (h[4] * h[8] - h[5] * h[7]) * id;
    hi[1] = (h[2] * h[7] - h[1] * h[8]) * id;
    hi[2] = (h[1] * h[5] - h[2] * h[4]) * id;
    hi[3] = (h[5] * h[6] - h[3] * h[8]) * id;
    hi[4] = (h[0] * h[8] - h[2] * h[6]) * id;
    hi[5] = (h[2] * h[3] - h[0] * h[5]) * id;
    hi[6] = (h[3] * h[7] - h[4] * h[6]) * id;
    hi[7] = (h[1] * h[6] - h[0] * h[7]) * id;
    hi[8] = (h[0] * h[4] - h[1] * h[3]) * id;
    return det;
}

// The same half-space set for a general cell: box rows are the lattice vectors a_d, the wave
// vectors k = 2 pi H^-1 n (k . a_d = 2 pi n_d, so |n_d| <= k_max |a_d| / 2 pi), V = |det H|.
// For fixed (n1, n2) the k with |k| < k_max form one run of n3 (|k|^2 is convex in n3).
inline KSet build_kset_box(const double box[9], double kmax, double alpha) {
    const double two_pi = 6.283185307179586;
    double hi[9];
    const double vol = std::fabs(invert3(box, hi));
    KSet ks;
    for (int d = 0; d < 3; ++d) {
        const double len = std::sqrt(box[3 * d] * box[3 * d] + box[3 * d + 1] * box[3 * d + 1] +
                                     box[3 * d + 2] * box[3 * d + 2]);
        ks.nmax[d] = (int)std::floor(kmax * len / two_pi);
    }
    auto k2_of = [&](int n1, int n2, int n3) {
        double k2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double kd = two_pi * (hi[3 * d] * n1 + hi[3 * d + 1] * n2 + hi[3 * d + 2] * n3);
            k2 += kd * kd;
        }
        return k2;
    };
    const int* nmax = ks.nmax;
    for (int n1 = 0; n1 <= nmax[0]; ++n1) {
        for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2) {
            if (n1 == 0 && n2 < 0) continue;
            int lo = 1 << 30, hi3 = -(1 << 30);
            for (int n3 = -nmax[2]; n3 <= nmax[2]; ++n3) {
                if (n1 == 0 && n2 == 0 && n3 <= 0) continue;
                const double k2 = k2_of(n1, n2, n3);
                if (k2 > 0 && k2 < kmax * kmax) {
                    lo = std::min(lo, n3);
                    hi3 = std::max(hi3, n3);
                }
            }
            if (hi3 < lo) continue;
            const int nchunk = (hi3 - lo + 1 + 7) / 8;
            const int c = (int)ks.cols.size();
            ks.cols.push_back(make_int4(n1, n2, lo, (int)ks.kg.size()));
            for (int h = 0; h < nchunk; ++h) ks.chunk_col.push_back(c);
            for (int t = 0; t < 8 * nchunk; ++t) {
                const int n3 = lo + t;
                const double k2 = k2_of(n1, n2, n3);
                const bool ok = n3 <= hi3 && k2 > 0 && k2 < kmax * kmax && !(n1 == 0 && n2 == 0 && n3 <= 0);
                ks.kg.push_back(ok ? (float)(two_pi / vol * std::exp(-k2 / (4 * alpha * alpha)) / k2) : 0.f);
            }
        }
    }
    ks.cols.push_back(make_int4(0, 0, 0, (int)ks.kg.size()));
    return ks;
}

}  // namespace qnep
