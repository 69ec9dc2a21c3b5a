// grid.cpp -- host-side FP64 construction of the radial and angular quadrature grids.
//
// Radial (Sec. II discretisation with Gauss-Legendre, Sec. III grids): u = ln s on
// [ln s_min, ln s_max] carries the Gauss-Legendre rule, so int ds s f(s) = int du s^2 f gives the
// weights W_j = (du/2) v_j s_j^2.  Collocated grids put the external points on the same nodes;
// staggered grids (the paper's modified interpolation, Eqs. pqrelationship and chazhiresult)
// put p_1 = s_min and ln p_i at the midpoints of consecutive internal nodes, so the bracket of
// q_j is known to be [p_j, p_{j+1}] without a search.
// Angular: Gauss-Chebyshev rule of the second kind for int_0^pi dtheta sin^2(theta) f(cos theta).
#include <cmath>
#include <vector>

#include "qdse_internal.h"

namespace qdse {

// Legendre P_n(x) and P_n'(x) by the Bonnet recurrence.
static void legendre_pd(int n, double x, double& p, double& dp) {
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    p = (n == 0) ? 1.0 : p1;
    dp = n * (p0 - x * p1) / (1.0 - x * x);  // P_n' = n (P_{n-1} - x P_n)/(1 - x^2)
}

// Gauss-Legendre nodes in ascending order and weights on [-1, 1].  Newton's method from
// Tricomi's asymptotic estimate of the k-th root.
int gauss_legendre_nodes(int n, double* t, double* v) {
    if (n < 1) return 1;
    for (int k = 1; k <= (n + 1) / 2; ++k) {
        double th = kPi * (4.0 * k - 1.0) / (4.0 * n + 2.0);
        double x = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) * std::cos(th);
        double p = 0, dp = 1;
        for (int it = 0; it < 50; ++it) {
            legendre_pd(n, x, p, dp);
            double dx = p / dp;
            x -= dx;
            if (std::fabs(dx) <= 1e-17) break;
        }
        legendre_pd(n, x, p, dp);
        double w = 2.0 / ((1.0 - x * x) * dp * dp);
        // root k counted from x = +1 downwards; mirror pair
        t[n - k] = x;
        v[n - k] = w;
        t[k - 1] = -x;
        v[k - 1] = w;
    }
    if (n % 2 == 1) t[n / 2] = 0.0;
    return 0;
}

void build_instance_grid(const qdse_grid& g, double* sp, double* sq, double* W, double* wt,
                         double* stc, int* sta) {
    const int n = g.n_p;
    std::vector<double> t(n), v(n), uq(n), up(n);
    gauss_legendre_nodes(n, t.data(), v.data());
    const double u0 = std::log(g.s_min), u1 = std::log(g.s_max);
    const double h = 0.5 * (u1 - u0), c = 0.5 * (u1 + u0);
    for (int j = 0; j < n; ++j) {
        uq[j] = c + h * t[j];
        sq[j] = std::exp(uq[j]);
        W[j] = h * v[j] * sq[j] * sq[j];
    }
    if (g.grid_mode == QDSE_STAGGERED) {
        up[0] = u0;
        sp[0] = g.s_min;
        for (int i = 1; i < n; ++i) {
            up[i] = 0.5 * (uq[i - 1] + uq[i]);
            sp[i] = std::exp(up[i]);
        }
    } else {
        for (int i = 0; i < n; ++i) {
            up[i] = uq[i];
            sp[i] = sq[i];
        }
    }
    // modified interpolation weights: F(q_j) = (1 - wt_j) F(p_j) + wt_j F(p_{j+1}), linear in |p|
    for (int j = 0; j < n; ++j) {
        if (g.grid_mode == QDSE_STAGGERED && j < n - 1) {
            double a = std::sqrt(sp[j]), b = std::sqrt(sp[j + 1]);
            wt[j] = (std::sqrt(sq[j]) - a) / (b - a);
        } else {
            wt[j] = 0.0;
        }
    }
    // collocated diagonal: dF/ds at p_i from the quadratic through three neighbours in u = ln s
    for (int i = 0; i < n; ++i) {
        int a = i - 1;
        if (a < 0) a = 0;
        if (a > n - 3) a = n - 3;
        const double x0 = up[a], x1 = up[a + 1], x2 = up[a + 2], x = up[i];
        const double c0 = ((x - x1) + (x - x2)) / ((x0 - x1) * (x0 - x2));
        const double c1 = ((x - x0) + (x - x2)) / ((x1 - x0) * (x1 - x2));
        const double c2 = ((x - x0) + (x - x1)) / ((x2 - x0) * (x2 - x1));
        sta[i] = a;
        stc[3 * i + 0] = c0 / sp[i];
        stc[3 * i + 1] = c1 / sp[i];
        stc[3 * i + 2] = c2 / sp[i];
    }
}

void build_angular(int nt, double* z, double* y, double* s2, double* w) {
    for (int k = 0; k < nt; ++k) {
        const double th = (k + 1) * kPi / (nt + 1);
        const double sn = std::sin(th), sh = std::sin(0.5 * th);
        z[k] = std::cos(th);
        y[k] = 2.0 * sh * sh;
        s2[k] = sn * sn;
        w[k] = kPi / (nt + 1) * sn * sn;
    }
}

}  // namespace qdse
