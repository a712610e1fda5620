// Host side of one column of a lock-step GMRES: the Hessenberg matrix of its
// Arnoldi process, reduced on the fly by complex Givens rotations (Saad and
// Schultz), the rotated right-hand side g = beta e_1, and the back
// substitution for the coefficients of the correction.  Real columns run
// through the same code with zero imaginary parts.
#pragma once

#include <cmath>
#include <vector>

namespace ibem {

struct GmresColumn {
    int m = 0;                     // restart length
    int k = 0;                     // Arnoldi steps taken in this cycle
    std::vector<double> H, g, cs, sr, si;

    void start(int restart, double beta) {
        m = restart;
        k = 0;
        H.assign((size_t)(m + 1) * m * 2, 0.0);
        g.assign(2 * (m + 1), 0.0);
        cs.assign(m, 0.0);
        sr.assign(m, 0.0);
        si.assign(m, 0.0);
        g[0] = beta;
    }
    double& hr(int i, int j) { return H[2 * ((size_t)i * m + j)]; }
    double& hi(int i, int j) { return H[2 * ((size_t)i * m + j) + 1]; }
    double hr(int i, int j) const { return H[2 * ((size_t)i * m + j)]; }
    double hi(int i, int j) const { return H[2 * ((size_t)i * m + j) + 1]; }

    // Column j of the Hessenberg matrix: h (complex, j + 1 entries, re/im
    // interleaved) and the norm hn of the orthogonalised vector.  Applies the
    // previous rotations, forms the new one and returns the residual estimate
    // |g_{j+1}|, or a negative value on breakdown.
    double add(int j, const double* h, double hn) {
        for (int i = 0; i <= j; ++i) {
            hr(i, j) = h[2 * i];
            hi(i, j) = h[2 * i + 1];
        }
        hr(j + 1, j) = hn;
        hi(j + 1, j) = 0.0;
        for (int i = 0; i < j; ++i) {
            const double ar = hr(i, j), ai = hi(i, j), br = hr(i + 1, j), bi = hi(i + 1, j);
            // [c s; -conj(s) c] with real c and complex s
            hr(i, j) = cs[i] * ar + (sr[i] * br - si[i] * bi);
            hi(i, j) = cs[i] * ai + (sr[i] * bi + si[i] * br);
            hr(i + 1, j) = -(sr[i] * ar + si[i] * ai) + cs[i] * br;
            hi(i + 1, j) = -(sr[i] * ai - si[i] * ar) + cs[i] * bi;
        }
        const double ar = hr(j, j), ai = hi(j, j), bb = hn;
        const double na = std::sqrt(ar * ar + ai * ai), den = std::sqrt(na * na + bb * bb);
        if (!(den > 0.0) || !std::isfinite(den)) return -1.0;
        if (na == 0.0) {
            cs[j] = 0.0;
            sr[j] = 1.0;
            si[j] = 0.0;
        } else {
            cs[j] = na / den;
            sr[j] = (ar / na) * bb / den;
            si[j] = (ai / na) * bb / den;
        }
        hr(j, j) = cs[j] * ar + sr[j] * bb;
        hi(j, j) = cs[j] * ai + si[j] * bb;
        hr(j + 1, j) = 0.0;
        hi(j + 1, j) = 0.0;
        const double gr = g[2 * j], gi = g[2 * j + 1];
        g[2 * j] = cs[j] * gr;
        g[2 * j + 1] = cs[j] * gi;
        g[2 * (j + 1)] = -(sr[j] * gr + si[j] * gi);
        g[2 * (j + 1) + 1] = -(sr[j] * gi - si[j] * gr);
        k = j + 1;
        const double res = std::hypot(g[2 * (j + 1)], g[2 * (j + 1) + 1]);
        return std::isfinite(res) ? res : -1.0;
    }

    // y (complex, k entries) with R y = g by back substitution
    void solve(std::vector<double>& y) const {
        y.assign(2 * k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            double s_r = g[2 * i], s_i = g[2 * i + 1];
            for (int l = i + 1; l < k; ++l) {
                s_r -= hr(i, l) * y[2 * l] - hi(i, l) * y[2 * l + 1];
                s_i -= hr(i, l) * y[2 * l + 1] + hi(i, l) * y[2 * l];
            }
            const double dr = hr(i, i), di = hi(i, i), den = dr * dr + di * di;
            y[2 * i] = (s_r * dr + s_i * di) / den;
            y[2 * i + 1] = (s_i * dr - s_r * di) / den;
        }
    }
};

}  // namespace ibem
