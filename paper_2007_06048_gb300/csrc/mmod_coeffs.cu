// Stencil weights of the Laplacian (Sec. 3): the order-8 Taylor weights, or
// weights that trade formal order for a smaller dispersion error.
//
// Optimised weights (host code): c_1..c_4 minimise
//     J(c) = int_0^kmax ( sum_m c_m a_m(k) - 1 )^2 dk,
//     a_m(k) = 2 (1 - cos(m k)) / k^2   (a_m(0) = m^2),
// the squared relative error of the 1-D second-derivative symbol over the band
// kh in [0, kmax], subject to sum_m m^2 c_m = 1 (exact on quadratics).  The
// constraint is eliminated, c = c_p + N y with c_p = g / |g|^2 and N an
// orthonormal basis of the plane g.c = 0 (Gram-Schmidt), and the remaining
// 3x3 normal equations are solved by Cholesky; the integrals use Simpson's
// rule on 2048 intervals.
#include <cmath>

#include "mmod_handle.h"

#define MMOD_API extern "C" __attribute__((visibility("default")))

namespace mmod {

namespace {

constexpr int kR = kRadius;

void symbol_terms(double k, double a[kR]) {
    for (int m = 1; m <= kR; ++m) {
        if (k < 1e-6) {   // series of 2(1 - cos mk)/k^2 near 0
            const double mk = m * k;
            a[m - 1] = (double)m * m * (1.0 - mk * mk / 12.0);
        } else {
            a[m - 1] = 2.0 * (1.0 - std::cos(m * k)) / (k * k);
        }
    }
}

}  // namespace

bool optimized_weights(double kmax, double c[kR]) {
    if (!(kmax > 0.0 && kmax <= M_PI)) return false;
    const double g[kR] = {1.0, 4.0, 9.0, 16.0};
    double gg = 0.0;
    for (double v : g) gg += v * v;
    double cp[kR];
    for (int m = 0; m < kR; ++m) cp[m] = g[m] / gg;
    // orthonormal basis of {x : g.x = 0}: Gram-Schmidt on the unit vectors
    double basis[kR][kR];
    int nb = 0;
    for (int e = 0; e < kR && nb < kR - 1; ++e) {
        double v[kR] = {0.0, 0.0, 0.0, 0.0};
        v[e] = 1.0;
        double pg = 0.0;
        for (int m = 0; m < kR; ++m) pg += v[m] * g[m];
        for (int m = 0; m < kR; ++m) v[m] -= pg * g[m] / gg;
        for (int b = 0; b < nb; ++b) {
            double p = 0.0;
            for (int m = 0; m < kR; ++m) p += v[m] * basis[b][m];
            for (int m = 0; m < kR; ++m) v[m] -= p * basis[b][m];
        }
        double nv = 0.0;
        for (int m = 0; m < kR; ++m) nv += v[m] * v[m];
        nv = std::sqrt(nv);
        if (nv < 1e-8) continue;
        for (int m = 0; m < kR; ++m) basis[nb][m] = v[m] / nv;
        ++nb;
    }
    if (nb != kR - 1) return false;
    // normal equations in y:  (N^T G N) y = N^T (b - G c_p),  G = int a a^T, b = int a
    constexpr int nint = 2048;
    double G[kR][kR] = {}, bv[kR] = {};
    for (int q = 0; q <= nint; ++q) {
        const double k = kmax * q / nint;
        const double w = (kmax / nint / 3.0) * ((q == 0 || q == nint) ? 1.0 : (q % 2 ? 4.0 : 2.0));
        double a[kR];
        symbol_terms(k, a);
        for (int i = 0; i < kR; ++i) {
            bv[i] += w * a[i];
            for (int j = 0; j < kR; ++j) G[i][j] += w * a[i] * a[j];
        }
    }
    constexpr int n = kR - 1;
    double H[n][n], r[n];
    for (int i = 0; i < n; ++i) {
        r[i] = 0.0;
        for (int p = 0; p < kR; ++p) {
            double Gcp_p = 0.0;
            for (int q = 0; q < kR; ++q) Gcp_p += G[p][q] * cp[q];
            r[i] += basis[i][p] * (bv[p] - Gcp_p);
        }
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int p = 0; p < kR; ++p)
                for (int q = 0; q < kR; ++q) s += basis[i][p] * G[p][q] * basis[j][q];
            H[i][j] = s;
        }
    }
    // Cholesky H = L L^T, then two triangular solves
    double L[n][n] = {};
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = H[i][j];
            for (int p = 0; p < j; ++p) s -= L[i][p] * L[j][p];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i][i] = std::sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    double z[n], y[n];
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int p = 0; p < i; ++p) s -= L[i][p] * z[p];
        z[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = z[i];
        for (int p = i + 1; p < n; ++p) s -= L[p][i] * y[p];
        y[i] = s / L[i][i];
    }
    for (int m = 0; m < kR; ++m) {
        c[m] = cp[m];
        for (int i = 0; i < n; ++i) c[m] += basis[i][m] * y[i];
    }
    return true;
}

double symbol_max(const double c[kR]) {
    // largest S(k) = sum_m 2 c_m (1 - cos m k) over [0, pi] (fine sampling;
    // the Taylor weights peak at k = pi with 2048/315)
    double best = 0.0;
    constexpr int ns = 8192;
    for (int q = 0; q <= ns; ++q) {
        const double k = M_PI * q / ns;
        double s = 0.0;
        for (int m = 1; m <= kR; ++m) s += 2.0 * c[m - 1] * (1.0 - std::cos(m * k));
        if (s > best) best = s;
    }
    return best;
}

void set_weights(mmod_handle *h, const double c[kR]) {
    const auto &cfg = h->cfg;
    for (int m = 0; m < kR; ++m) {
        h->coef[m] = c[m];
        h->w.x[m] = (float)(c[m] / (cfg.hx * cfg.hx));
        h->w.y[m] = (float)(c[m] / (cfg.hy * cfg.hy));
        h->w.z[m] = (float)(c[m] / (cfg.hz * cfg.hz));
    }
    h->symbol_max = symbol_max(c);
}

}  // namespace mmod

MMOD_API mmod_status mmod_optimized_coefficients(double kmax, double *c4) {
    if (!c4) return MMOD_ERR_ARG;
    return mmod::optimized_weights(kmax, c4) ? MMOD_OK : MMOD_ERR_ARG;
}

MMOD_API mmod_status mmod_set_fd_coefficients(mmod_handle *h, const double *c4) {
    if (!h) return MMOD_ERR_ARG;
    double c[mmod::kR];
    if (c4) {
        double s = 0.0;
        for (int m = 0; m < mmod::kR; ++m) {
            if (!std::isfinite(c4[m])) return mmod::fail(h, MMOD_ERR_ARG, "coefficients must be finite");
            c[m] = c4[m];
            s += (double)(m + 1) * (m + 1) * c4[m];
        }
        if (std::fabs(s - 1.0) > 1e-6)
            return mmod::fail(h, MMOD_ERR_ARG, "coefficients must satisfy sum m^2 c_m = 1 (consistency)");
        if (!(mmod::symbol_max(c) > 0.0)) return mmod::fail(h, MMOD_ERR_ARG, "coefficients give no stable step");
    } else {
        for (int m = 0; m < mmod::kR; ++m) c[m] = mmod::kTaylor8[m];
    }
    mmod::set_weights(h, c);
    mmod::drop_graphs(h);   // captured steps hold the old weights
    if (h->model_set) {     // the stability bound depends on the weights
        const double ksum = h->symbol_max * (1.0 / (h->cfg.hx * h->cfg.hx) + 1.0 / (h->cfg.hy * h->cfg.hy) +
                                             1.0 / (h->cfg.hz * h->cfg.hz));
        if (h->cfg.dt * h->vmax * std::sqrt(ksum) > 2.0) {
            h->model_set = false;
            return mmod::fail(h, MMOD_ERR_UNSTABLE, "dt too large for the model with these coefficients");
        }
    }
    return MMOD_OK;
}
