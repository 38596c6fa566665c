// Least-squares fit of the 27-point mixed-grid stencil weights.
//
// The paper computes the stiffness and consistent-mass weights by least
// squares on the numerical dispersion and anisotropy without printing them.
// Objective here: the normalised phase-velocity error
//   e(G, n) = 1 - sqrt(-L(kappa)/M(kappa)) / |kappa|,  kappa = (2 pi / G) n  (h = 1)
// with L, M the Laplacian and mass symbols of the product form
//   L = sum s + a2 sum s_a s_b + a3 s_x s_y s_z,
//   M = m0 + m1 sum s + m2 sum s_a s_b + m3 s_x s_y s_z,  s_a = 2 (cos kappa_a - 1),
// sampled at 24 values of 1/G evenly spaced in [1/G_max, 1/G_min] and 7 x 7
// directions in one octant.  Free parameters (w2, w3, wm2, wm3, wm4) within
// non-negative bounds; w1 and wm1 follow from the sum-to-one constraints.
// Solved by a projected Levenberg-Marquardt iteration.
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/helm.h"

namespace {

void full(const double* p, double* w) {
    w[0] = 1.0 - p[0] - p[1];
    w[1] = p[0];
    w[2] = p[1];
    w[3] = 1.0 - 6.0 * p[2] - 12.0 * p[3] - 8.0 * p[4];
    w[4] = p[2];
    w[5] = p[3];
    w[6] = p[4];
}

struct Sample {
    double G, n[3];
};

void residuals(const double* p, const std::vector<Sample>& S, std::vector<double>& r) {
    double w[7];
    full(p, w);
    const double a2 = w[1] / 6.0 + w[2] / 2.0, a3 = w[2] / 4.0;
    const double m0 = w[3] + 6 * w[4] + 12 * w[5] + 8 * w[6], m1 = w[4] + 4 * w[5] + 4 * w[6],
                 m2 = w[5] + 2 * w[6], m3 = w[6];
    r.resize(S.size());
    for (size_t q = 0; q < S.size(); ++q) {
        const double kap = 2.0 * M_PI / S[q].G;
        double s[3];
        for (int a = 0; a < 3; ++a) s[a] = 2.0 * (cos(kap * S[q].n[a]) - 1.0);
        const double s1 = s[0] + s[1] + s[2], s2 = s[0] * s[1] + s[0] * s[2] + s[1] * s[2], s3 = s[0] * s[1] * s[2];
        const double L = s1 + a2 * s2 + a3 * s3, M = m0 + m1 * s1 + m2 * s2 + m3 * s3;
        const double ratio = -L / M;
        r[q] = 1.0 - sqrt(ratio > 0 ? ratio : 0.0) / kap;
    }
}

double cost(const std::vector<double>& r) {
    double c = 0;
    for (double v : r) c += v * v;
    return c;
}

// Solve the 5x5 symmetric system A x = b by Gaussian elimination with partial pivoting.
bool solve5(double A[5][5], double b[5], double x[5]) {
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int r = c + 1; r < 5; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (fabs(A[piv][c]) < 1e-300) return false;
        if (piv != c) {
            for (int k = 0; k < 5; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < 5; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 5; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = 4; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 5; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return true;
}

}  // namespace

extern "C" helm_status helm_fit_weights(double G_min, double G_max, double* out) {
    if (!out || !(G_min >= 2.0) || !(G_max > G_min)) return HELM_EINVAL;
    std::vector<Sample> S;
    for (int g = 0; g < 24; ++g) {
        const double inv = 1.0 / G_max + (1.0 / G_min - 1.0 / G_max) * g / 23.0;
        for (int t = 0; t < 7; ++t)
            for (int f = 0; f < 7; ++f) {
                const double th = 0.5 * M_PI * t / 6.0, ph = 0.5 * M_PI * f / 6.0;
                S.push_back({1.0 / inv, {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)}});
            }
    }
    const double lo[5] = {0, 0, 0, 0, 0};
    const double hi[5] = {1.0, 1.0, 1.0 / 6.0, 1.0 / 12.0, 1.0 / 8.0};
    double p[5] = {0.5, 0.1, 0.08, 0.005, 0.001};
    std::vector<double> r, rp, J(5 * 0);
    residuals(p, S, r);
    double c = cost(r), lambda = 1e-3;
    const size_t M = S.size();
    J.resize(5 * M);
    for (int it = 0; it < 500; ++it) {
        for (int a = 0; a < 5; ++a) {
            double q[5];
            memcpy(q, p, sizeof q);
            const double step = 1e-7 * (fabs(p[a]) + 1e-3);
            q[a] += step;
            residuals(q, S, rp);
            for (size_t m = 0; m < M; ++m) J[a * M + m] = (rp[m] - r[m]) / step;
        }
        double JTJ[5][5], g[5];
        for (int a = 0; a < 5; ++a) {
            g[a] = 0;
            for (size_t m = 0; m < M; ++m) g[a] += J[a * M + m] * r[m];
            for (int b = 0; b < 5; ++b) {
                double s = 0;
                for (size_t m = 0; m < M; ++m) s += J[a * M + m] * J[b * M + m];
                JTJ[a][b] = s;
            }
        }
        bool improved = false;
        for (int tries = 0; tries < 30 && !improved; ++tries) {
            double A[5][5], b[5], dx[5] = {0, 0, 0, 0, 0};
            for (int a = 0; a < 5; ++a) {
                for (int k = 0; k < 5; ++k) A[a][k] = JTJ[a][k];
                A[a][a] += lambda * (JTJ[a][a] + 1e-12);
                b[a] = -g[a];
            }
            if (!solve5(A, b, dx)) { lambda *= 10; continue; }
            double q[5];
            for (int a = 0; a < 5; ++a) q[a] = fmin(hi[a], fmax(lo[a], p[a] + dx[a]));
            residuals(q, S, rp);
            const double cq = cost(rp);
            if (cq < c) {
                const double rel = (c - cq) / c;
                memcpy(p, q, sizeof p);
                r = rp;
                c = cq;
                lambda = fmax(lambda * 0.3, 1e-12);
                improved = true;
                if (rel < 1e-13) it = 1 << 20;
            } else {
                lambda *= 10;
            }
        }
        if (!improved) break;
    }
    full(p, out);
    return HELM_OK;
}
