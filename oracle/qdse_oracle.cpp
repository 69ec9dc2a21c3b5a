/*
 * qdse_oracle.cpp -- plain, slow FP64 CPU oracle for the vacuum quark gap equation with the
 * Ball-Chiu (BC) vertex (Huang, Duan, Hu, Chen, arXiv:2012.03667).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the GPU solver.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant generator with the CUDA path, and it never reads anything the
 * CUDA path produced.
 *
 * What it computes (paper section II):
 *   gap equation            S^-1(p) = i g.p A(p^2) + B(p^2)                  (Eq. gendse, Sec. II)
 *   truncation              G(k^2) D0_{rho sigma}(k) (lambda^a/2) Gamma_sigma (Eq. KernelAnsatz)
 *   interaction             D(k^2) = 8 pi^2 D / w^4 exp(-k^2/w^2)            (Eq. IRGsQC)
 *   BC vertex               Gamma = Sigma_A g_mu + 1/2 t_mu g.t Delta_A - i t_mu Delta_B
 *                                                                             (Eq. bcvtxmu, Eq. 2)
 *   projected equations     A = 1 + ..., B = m + ...                          (Eqs. dsesys, dsesys2)
 *   successive approximation u_{n+1} = f + int K F(u_n)                      (Eqs. jifen14-jifen122)
 *   stopping rule           change at every point below the tolerance        (Eq. jifenab2)
 *   modified interpolation  interleaved p/q grids                            (Eqs. pqrelationship,
 *                                                                              chazhiresult)
 *
 * Readings of the paper taken here (the paper is garbled or silent at these places):
 *   R1  the denominator is the internal propagator d_q = Q A(Q)^2 + B(Q)^2 (S(q) is inside the
 *       integral of Eq. gendse).
 *   R2  the factor multiplying the transverse projector is 8 pi^2 D/w^4 exp(-k^2/w^2): the
 *       1/k^2 of D0 is absorbed (the Qin-Chang convention G(s)/s); with the paper's D, w this
 *       gives D w = 0.373 GeV^3, the standard value.
 *   R3  the A-projection carries a single 1/P (projection tr[-i g.p Sigma]/(4P)).
 *   R4  lambda_1 = Sigma_A = (A(p^2) + A(q^2))/2, as the Ward-Takahashi identity requires.
 *   R5  colour factor C_F = 4/3 from lambda^a/2 ... lambda^a/2 (configurable).
 *   R6  Jacobi sweeps: every new A_i, B_i is computed from the previous iterate only.
 *   R7  stopping rule |x_new - x_old| <= tol * max(|x_new|, floor), floor_A = 0,
 *       floor_B = 1e-12 max_j |B_j|, 0/0 counts as converged.
 *   R8  on a collocated grid the diagonal q^2 = p^2 uses dF/ds from the derivative of the
 *       3-point Lagrange polynomial in u = ln s (one-sided at the ends).
 *   R9  modified interpolation is linear in |p|; F(q_N) = F(p_N).
 *   R10 angular rule: Gauss-Chebyshev of the second kind (weight sin^2 theta).
 *   R15 the traditional interpolation of Table 1 (algorithms 1, 3) searches the external grid
 *       linearly for q's bracket at every integrand evaluation, then applies Eq. chazhiresult0;
 *       grid_mode 2 selects it (timing only: the values equal those of grid_mode 1).
 *
 * After the Dirac traces the per-point integrand reduces to three angular kernels
 *   g_T = 2 P Q (1 - z^2) / k^2,   g_3 = [3 x (P+Q) - 4 x^2 - 2 P Q] / k^2,   g_0 = 1
 * (x = sqrt(PQ) z, k = p - q):
 *   I_A = [ -B_q Delta_B g_T - 1/2 A_q Delta_A (P+Q) g_T + A_q Sigma_A g_3 ] / (P d_q)
 *   I_B = [ -A_q Delta_B g_T + B_q Delta_A g_T + 3 B_q Sigma_A ] / d_q
 * and A_i = 1 + C_F/(8 pi^3) sum_j W_j sum_k w_k D(k^2) I_A,  B_i = m + (same with I_B).
 * The test-suite pins this reduction against explicit 4x4 Euclidean gamma-matrix traces.
 *
 * Everything is evaluated straight from these definitions, one (i, j, k) triple at a time, with
 * no precomputation of angular kernel matrices.  The sweep is templated on the scalar type so
 * that the same code runs in std::complex<double> for complex-step derivatives.
 */
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::complex<double> cplx;

const double kPi = 3.14159265358979323846264338327950288;

/* Plain configuration of one instance. */
struct Cfg {
    int n;          /* radial points (external = internal count)            */
    int n_theta;    /* angular nodes                                         */
    double s_min, s_max; /* GeV^2                                            */
    int grid_mode;  /* 0 collocated, 1 staggered (modified interpolation)    */
    int traditional; /* staggered, bracket found at every evaluation (R15)   */
    int vertex;     /* 0 Ball-Chiu, 1 rainbow (bare vertex)                  */
    double cf;      /* colour factor                                         */
};

/* ---------------------------------------------------------------------------------------- */
/* Quadrature.                                                                              */
/* ---------------------------------------------------------------------------------------- */

/* P_n(x) by the three-term recurrence and P_n'(x) = n (x P_n - P_{n-1})/(x^2 - 1). */
void legendre(int n, double x, double* pn_out, double* dp_out) {
    double pm = 1.0, pn = x;                    /* P_0, P_1 */
    for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * pn - (k - 1.0) * pm) / k;
        pm = pn;
        pn = pk;
    }
    *pn_out = pn;
    *dp_out = n * (x * pn - pm) / (x * x - 1.0);
}

/* Gauss-Legendre nodes t (ascending) and weights v on [-1, 1]: Newton iteration on the Legendre
 * polynomial P_n from the Chebyshev-like initial guess cos(pi (i - 1/4)/(n + 1/2)). */
int gauss_legendre(int n, double* t, double* v) {
    if (n < 1) return 1;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double pn = 0.0, dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            legendre(n, x, &pn, &dp);
            double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        legendre(n, x, &pn, &dp);
        t[n - 1 - i] = x;                       /* ascending order */
        v[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return 0;
}

/* Radial grids.  u = ln s is the GL variable mapped onto [ln s_min, ln s_max].
 * The measure  int ds s f(s) = int du s^2 f  gives W_j = (du/2) v_j s_j^2.
 *   collocated : q-grid = p-grid = the GL nodes.
 *   staggered  : q-grid = the GL nodes; p_1 = s_min, u^p_i = (u^q_{i-1} + u^q_i)/2, so that
 *                p_1 < q_1 < p_2 < ... < p_N < q_N (Eq. pqrelationship). */
int radial_grid(const Cfg& c, double* sp, double* sq, double* W) {
    const int n = c.n;
    std::vector<double> t(n), v(n);
    if (gauss_legendre(n, t.data(), v.data())) return 1;
    const double umin = std::log(c.s_min), umax = std::log(c.s_max);
    const double half = 0.5 * (umax - umin), mid = 0.5 * (umax + umin);
    std::vector<double> uq(n);
    for (int j = 0; j < n; ++j) {
        uq[j] = mid + half * t[j];
        sq[j] = std::exp(uq[j]);
        W[j] = half * v[j] * sq[j] * sq[j];
    }
    if (c.grid_mode == 0) {
        for (int i = 0; i < n; ++i) sp[i] = sq[i];
    } else {
        sp[0] = c.s_min;
        for (int i = 1; i < n; ++i) sp[i] = std::exp(0.5 * (uq[i - 1] + uq[i]));
    }
    return 0;
}

/* Gauss-Chebyshev rule of the second kind on theta in (0, pi):
 *   int_0^pi dtheta sin^2(theta) f(cos theta) ~ sum_k w_k f(z_k),
 *   theta_k = k pi/(M+1), z_k = cos theta_k, w_k = pi/(M+1) sin^2 theta_k, k = 1..M.
 * y_k = 1 - z_k = 2 sin^2(theta_k/2) is returned separately (no cancellation near z = 1). */
void angular_grid(int m, double* z, double* y, double* w) {
    for (int k = 1; k <= m; ++k) {
        double th = k * kPi / (m + 1);
        double sh = std::sin(0.5 * th);
        z[k - 1] = std::cos(th);
        y[k - 1] = 2.0 * sh * sh;
        w[k - 1] = kPi / (m + 1) * std::sin(th) * std::sin(th);
    }
}

/* "Traditional" interpolation bracket: search the external grid for p[b] <= q < p[b+1]
 * (the paper's finding step before Eq. chazhiresult0).  Returns n-1 when q >= p[n-1]. */
int find_bracket(const double* sp, int n, double q) {
    int lo = 0, hi = n - 1;
    if (q >= sp[n - 1]) return n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (sp[mid] <= q) lo = mid; else hi = mid;
    }
    return lo;
}

/* Derivative at u_a of the quadratic Lagrange interpolant through (u_l, f_l), l = 0,1,2. */
template <class T>
T lagrange3_deriv(const double u[3], const T f[3], double ua) {
    T d = T(0.0);
    for (int l = 0; l < 3; ++l) {
        double num = 0.0, den = 1.0;
        for (int m = 0; m < 3; ++m) {
            if (m == l) continue;
            den *= (u[l] - u[m]);
            double prod = 1.0;
            for (int r = 0; r < 3; ++r) if (r != l && r != m) prod *= (ua - u[r]);
            num += prod;
        }
        d += f[l] * (num / den);
    }
    return d;
}

/* dF/ds at node i of a collocated grid (reading R8). */
template <class T>
T diag_quotient(const double* s, int n, const T* F, int i) {
    int a = i - 1;
    if (a < 0) a = 0;
    if (a > n - 3) a = n - 3;
    double u[3] = {std::log(s[a]), std::log(s[a + 1]), std::log(s[a + 2])};
    T f[3] = {F[a], F[a + 1], F[a + 2]};
    return lagrange3_deriv(u, f, std::log(s[i])) / s[i];
}

/* ---------------------------------------------------------------------------------------- */
/* Point integrand of Eqs. dsesys/dsesys2 after the traces (without interaction and measure). */
/* ---------------------------------------------------------------------------------------- */
template <class T>
void point_integrand(double P, double Q, double z, T Ap, T Bp, T Aq, T Bq, T DA, T DB,
                     double k2, int vertex, T* IA, T* IB) {
    const double x = std::sqrt(P * Q) * z;
    const double gT = 2.0 * (P * Q - x * x) / k2;
    const double g3 = (3.0 * x * (P + Q) - 4.0 * x * x - 2.0 * P * Q) / k2;
    (void)Bp;  /* B(p^2) enters only through Delta_B */
    const T dq = Q * Aq * Aq + Bq * Bq;
    T SA = 0.5 * (Ap + Aq);
    if (vertex == 1) { SA = T(1.0); DA = T(0.0); DB = T(0.0); }
    /* the six I-terms of Eq. dsesys2 in reduced form */
    T IA1 = -Bq * DB * gT / P;
    T IA2 = -0.5 * Aq * DA * (P + Q) * gT / P;
    T IA3 = Aq * SA * g3 / P;
    T IB1 = -Aq * DB * gT;
    T IB2 = 3.0 * Bq * SA;
    T IB3 = Bq * DA * gT;
    *IA = (IA1 + IA2 + IA3) / dq;
    *IB = (IB1 + IB2 + IB3) / dq;
}

/* Grid bundle for one instance. */
struct Grid {
    std::vector<double> sp, sq, W, z, y, w;
    std::vector<int> br;  /* staggered: bracket of q_j on the p grid (traditional search) */
};

int build_grid(const Cfg& c, Grid& g) {
    if (c.n < 3 || c.n_theta < 1 || !(c.s_min > 0) || !(c.s_max > c.s_min)) return 1;
    g.sp.resize(c.n); g.sq.resize(c.n); g.W.resize(c.n);
    g.z.resize(c.n_theta); g.y.resize(c.n_theta); g.w.resize(c.n_theta);
    if (radial_grid(c, g.sp.data(), g.sq.data(), g.W.data())) return 1;
    angular_grid(c.n_theta, g.z.data(), g.y.data(), g.w.data());
    g.br.resize(c.n);
    for (int j = 0; j < c.n; ++j) g.br[j] = find_bracket(g.sp.data(), c.n, g.sq[j]);
    return 0;
}

/* Values of A or B at the internal node q_j. */
template <class T>
T at_q(const Cfg& c, const Grid& g, const T* F, int j) {
    if (c.grid_mode == 0) return F[j];
    int b = g.br[j];
    if (b >= c.n - 1) return F[c.n - 1];                         /* F(q_N) = F(p_N) */
    double pb = std::sqrt(g.sp[b]), pb1 = std::sqrt(g.sp[b + 1]), q = std::sqrt(g.sq[j]);
    return F[b] + (q - pb) * (F[b + 1] - F[b]) / (pb1 - pb);     /* Eq. chazhiresult */
}

/* Reading R15, the paper's traditional interpolation (Sec. III; Table 1, algorithms 1 and 3):
 * no bracket is kept between evaluations; each one scans the external grid for
 * p[b] <= q < p[b+1] (the finding step before Eq. chazhiresult0) and interpolates there.  The
 * values equal at_q's exactly; only the work differs.  noipa keeps the compiler from proving the
 * call loop-invariant and hoisting the search out of the angular loop. */
__attribute__((noipa)) double at_q_traditional(const Cfg& c, const Grid& g, const double* F,
                                                int j) {
    const double q2 = g.sq[j];
    int b = 0;
    while (b + 1 < c.n && g.sp[b + 1] <= q2) ++b;
    if (b >= c.n - 1) return F[c.n - 1];
    const double pb = std::sqrt(g.sp[b]), pb1 = std::sqrt(g.sp[b + 1]), q = std::sqrt(q2);
    return F[b] + (q - pb) * (F[b + 1] - F[b]) / (pb1 - pb);
}

template <class T>
void traditional_values(const Cfg&, const Grid&, const T*, const T*, int, T*, T*) {}
template <>
void traditional_values<double>(const Cfg& c, const Grid& g, const double* A, const double* B,
                                int j, double* Aq, double* Bq) {
    *Aq = at_q_traditional(c, g, A, j);
    *Bq = at_q_traditional(c, g, B, j);
}

/* One Jacobi sweep  x_{n+1} = F(x_n)  for external rows [i0, i1).  Plain triple loop. */
template <class T>
void sweep_rows(const Cfg& c, const Grid& g, T D, T omega, T m, const T* A, const T* B,
                T* Aout, T* Bout, int i0, int i1) {
    const int n = c.n;
    const T pref = 8.0 * kPi * kPi * D / (omega * omega * omega * omega);
    const double meas = c.cf / (8.0 * kPi * kPi * kPi);
    for (int i = i0; i < i1; ++i) {
        const double P = g.sp[i];
        T SA = T(0.0), SB = T(0.0);
        for (int j = 0; j < n; ++j) {
            const double Q = g.sq[j];
            T Aq = at_q(c, g, A, j), Bq = at_q(c, g, B, j);
            T DA, DB;
            if (Q == P) {  /* collocated diagonal: removable limit (reading R8) */
                DA = diag_quotient(g.sp.data(), n, A, i);
                DB = diag_quotient(g.sp.data(), n, B, i);
            } else {
                DA = (Aq - A[i]) / (Q - P);
                DB = (Bq - B[i]) / (Q - P);
            }
            const double sP = std::sqrt(P), sQ = std::sqrt(Q);
            for (int k = 0; k < c.n_theta; ++k) {
                if (c.traditional) {  /* R15: interpolate again at every evaluation */
                    traditional_values<T>(c, g, A, B, j, &Aq, &Bq);
                    DA = (Aq - A[i]) / (Q - P);
                    DB = (Bq - B[i]) / (Q - P);
                }
                const double k2 = (sP - sQ) * (sP - sQ) + 2.0 * sP * sQ * g.y[k];
                const T Dk = pref * std::exp(-k2 / (omega * omega));
                T IA, IB;
                point_integrand<T>(P, Q, g.z[k], A[i], B[i], Aq, Bq, DA, DB, k2, c.vertex, &IA, &IB);
                SA += g.W[j] * g.w[k] * Dk * IA;
                SB += g.W[j] * g.w[k] * Dk * IB;
            }
        }
        Aout[i] = 1.0 + meas * SA;
        Bout[i] = m + meas * SB;
    }
}

template <class T>
void sweep(const Cfg& c, const Grid& g, T D, T omega, T m, const T* A, const T* B, T* Aout,
           T* Bout, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 1) {
        /* the paper's Listing-2 scheme: parallel for over the external index */
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
        for (int i = 0; i < c.n; ++i) sweep_rows<T>(c, g, D, omega, m, A, B, Aout, Bout, i, i + 1);
        return;
    }
#endif
    (void)nthreads;
    sweep_rows<T>(c, g, D, omega, m, A, B, Aout, Bout, 0, c.n);
}

/* Reading R7. */
double max_rel_change(int n, const double* Aold, const double* Bold, const double* Anew,
                      const double* Bnew) {
    double bmax = 0.0;
    for (int i = 0; i < n; ++i) bmax = std::fmax(bmax, std::fabs(Bnew[i]));
    const double floorB = 1e-12 * bmax;
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
        double da = std::fabs(Anew[i] - Aold[i]), na = std::fabs(Anew[i]);
        double db = std::fabs(Bnew[i] - Bold[i]), nb = std::fmax(std::fabs(Bnew[i]), floorB);
        double ra = (da == 0.0) ? 0.0 : (na > 0.0 ? da / na : INFINITY);
        double rb = (db == 0.0) ? 0.0 : (nb > 0.0 ? db / nb : INFINITY);
        if (!(ra <= r)) r = std::isnan(ra) ? NAN : std::fmax(r, ra);
        if (!(rb <= r)) r = std::isnan(rb) ? NAN : std::fmax(r, rb);
        if (std::isnan(r)) return NAN;
    }
    return r;
}

/* Dense LU with partial pivoting, solving M x = b in place (b overwritten). */
int lu_solve(int n, std::vector<double>& M, double* b) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(M[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = std::fabs(M[(size_t)r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return 1;
        if (p != k) {
            for (int cidx = 0; cidx < n; ++cidx)
                std::swap(M[(size_t)k * n + cidx], M[(size_t)p * n + cidx]);
            std::swap(b[k], b[p]);
        }
        for (int r = k + 1; r < n; ++r) {
            double f = M[(size_t)r * n + k] / M[(size_t)k * n + k];
            if (f == 0.0) continue;
            for (int cidx = k; cidx < n; ++cidx) M[(size_t)r * n + cidx] -= f * M[(size_t)k * n + cidx];
            b[r] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int cidx = k + 1; cidx < n; ++cidx) s -= M[(size_t)k * n + cidx] * b[cidx];
        b[k] = s / M[(size_t)k * n + k];
    }
    return 0;
}

Cfg make_cfg(int n, int n_theta, double s_min, double s_max, int grid_mode, int vertex, double cf) {
    Cfg c;
    c.n = n; c.n_theta = n_theta; c.s_min = s_min; c.s_max = s_max;
    c.grid_mode = grid_mode == 2 ? 1 : grid_mode; c.vertex = vertex; c.cf = cf;
    c.traditional = grid_mode == 2;
    return c;
}

}  // namespace

/* ---------------------------------------------------------------------------------------- */
/* C interface used by oracle/oracle.py                                                      */
/* ---------------------------------------------------------------------------------------- */
extern "C" {

int oracle_gauss_legendre(int n, double* t, double* v) { return gauss_legendre(n, t, v); }

void oracle_angular_grid(int m, double* z, double* y, double* w) { angular_grid(m, z, y, w); }

/* Radial grid: sp (external), sq (internal), W (internal weights), bracket (staggered). */
int oracle_radial_grid(int n, double s_min, double s_max, int grid_mode, double* sp, double* sq,
                       double* W, int* bracket) {
    Cfg c = make_cfg(n, 1, s_min, s_max, grid_mode, 0, 4.0 / 3.0);
    Grid g;
    if (build_grid(c, g)) return 1;
    for (int j = 0; j < n; ++j) {
        sp[j] = g.sp[j]; sq[j] = g.sq[j]; W[j] = g.W[j];
        if (bracket) bracket[j] = g.br[j];
    }
    return 0;
}

/* Values of F at the internal nodes: on-grid (collocated) or the modified interpolation of
 * Eq. chazhiresult on the staggered grid. */
int oracle_values_at_q(int n, double s_min, double s_max, int grid_mode, const double* F,
                       double* Fq) {
    Cfg c = make_cfg(n, 1, s_min, s_max, grid_mode, 0, 4.0 / 3.0);
    Grid g;
    if (build_grid(c, g)) return 1;
    for (int j = 0; j < n; ++j) Fq[j] = at_q<double>(c, g, F, j);
    return 0;
}

/* Reduced integrand at one point (no interaction factor, no measure). */
void oracle_point_integrand(double P, double Q, double z, double Ap, double Bp, double Aq,
                            double Bq, double DA, double DB, int vertex, double* IA, double* IB) {
    const double sP = std::sqrt(P), sQ = std::sqrt(Q);
    const double k2 = (sP - sQ) * (sP - sQ) + 2.0 * sP * sQ * (1.0 - z);
    point_integrand<double>(P, Q, z, Ap, Bp, Aq, Bq, DA, DB, k2, vertex, IA, IB);
}

/* Derivative dF/ds at node i from the 3-point Lagrange stencil in ln s (reading R8). */
double oracle_diag_quotient(const double* s, int n, const double* F, int i) {
    return diag_quotient<double>(s, n, F, i);
}

/* One Jacobi sweep. */
int oracle_sweep(int n, int n_theta, double s_min, double s_max, int grid_mode, int vertex,
                 double cf, double D, double omega, double m, const double* A, const double* B,
                 double* Aout, double* Bout, int nthreads) {
    Cfg c = make_cfg(n, n_theta, s_min, s_max, grid_mode, vertex, cf);
    Grid g;
    if (build_grid(c, g)) return 1;
    sweep<double>(c, g, D, omega, m, A, B, Aout, Bout, nthreads);
    return 0;
}

/* Successive approximation to the R7 tolerance.  A, B hold the start on entry and the last
 * iterate on exit.  Returns 0 converged, 4 not converged, 5 non-finite, 1 bad argument. */
int oracle_solve(int n, int n_theta, double s_min, double s_max, int grid_mode, int vertex,
                 double cf, double D, double omega, double m, double tol, double alpha,
                 int max_iter, double* A, double* B, int* iters, double* last_change,
                 int nthreads) {
    Cfg c = make_cfg(n, n_theta, s_min, s_max, grid_mode, vertex, cf);
    Grid g;
    if (build_grid(c, g)) return 1;
    std::vector<double> An(n), Bn(n);
    int it = 0;
    double ch = INFINITY;
    int status = 4;
    while (it < max_iter) {
        sweep<double>(c, g, D, omega, m, A, B, An.data(), Bn.data(), nthreads);
        for (int i = 0; i < n; ++i) {
            An[i] = (1.0 - alpha) * A[i] + alpha * An[i];
            Bn[i] = (1.0 - alpha) * B[i] + alpha * Bn[i];
        }
        ch = max_rel_change(n, A, B, An.data(), Bn.data());
        std::memcpy(A, An.data(), sizeof(double) * n);
        std::memcpy(B, Bn.data(), sizeof(double) * n);
        ++it;
        if (std::isnan(ch) || std::isinf(ch)) { status = 5; break; }
        if (ch <= tol) { status = 0; break; }
    }
    if (iters) *iters = it;
    if (last_change) *last_change = ch;
    return status;
}

/* Jacobian of the sweep map F at x = (A, B) by the complex step:  J e_c = Im F(x + i h e_c)/h.
 * J is 2n x 2n row-major, rows/columns ordered (A_0..A_{n-1}, B_0..B_{n-1}). */
int oracle_jacobian(int n, int n_theta, double s_min, double s_max, int grid_mode, int vertex,
                    double cf, double D, double omega, double m, const double* A, const double* B,
                    double* J, int nthreads) {
    Cfg c = make_cfg(n, n_theta, s_min, s_max, grid_mode, vertex, cf);
    Grid g;
    if (build_grid(c, g)) return 1;
    const double h = 1e-30;
    const int nn = 2 * n;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 1)
#endif
    for (int col = 0; col < nn; ++col) {
        std::vector<cplx> Ac(n), Bc(n), Ao(n), Bo(n);
        for (int i = 0; i < n; ++i) { Ac[i] = cplx(A[i], 0.0); Bc[i] = cplx(B[i], 0.0); }
        if (col < n) Ac[col] += cplx(0.0, h); else Bc[col - n] += cplx(0.0, h);
        sweep_rows<cplx>(c, g, cplx(D), cplx(omega), cplx(m), Ac.data(), Bc.data(), Ao.data(),
                         Bo.data(), 0, n);
        for (int i = 0; i < n; ++i) {
            J[(size_t)i * nn + col] = Ao[i].imag() / h;
            J[(size_t)(n + i) * nn + col] = Bo[i].imag() / h;
        }
    }
    (void)nthreads;
    return 0;
}

/* Derivatives of F with respect to theta = (m, D, omega) at fixed x, by the complex step.
 * dF is 3 x 2n row-major (row t = d F / d theta_t). */
int oracle_param_jacobian(int n, int n_theta, double s_min, double s_max, int grid_mode,
                          int vertex, double cf, double D, double omega, double m,
                          const double* A, const double* B, double* dF) {
    Cfg c = make_cfg(n, n_theta, s_min, s_max, grid_mode, vertex, cf);
    Grid g;
    if (build_grid(c, g)) return 1;
    const double h = 1e-30;
    std::vector<cplx> Ac(n), Bc(n), Ao(n), Bo(n);
    for (int i = 0; i < n; ++i) { Ac[i] = cplx(A[i], 0.0); Bc[i] = cplx(B[i], 0.0); }
    for (int t = 0; t < 3; ++t) {
        cplx mc(m), Dc(D), wc(omega);
        if (t == 0) mc += cplx(0.0, h);
        if (t == 1) Dc += cplx(0.0, h);
        if (t == 2) wc += cplx(0.0, h);
        sweep_rows<cplx>(c, g, Dc, wc, mc, Ac.data(), Bc.data(), Ao.data(), Bo.data(), 0, n);
        for (int i = 0; i < n; ++i) {
            dF[(size_t)t * 2 * n + i] = Ao[i].imag() / h;
            dF[(size_t)t * 2 * n + n + i] = Bo[i].imag() / h;
        }
    }
    return 0;
}

/* Adjoint at a converged x* = F(x*):  solve (I - J^T) lambda = g  by dense LU, then
 * dL/dtheta = lambda^T dF/dtheta for theta = (m, D, omega, mu).  In the vacuum equation mu does
 * not enter, so its entry is 0.  g = (gA, gB); lambda (2n) is returned if non-null. */
int oracle_adjoint(int n, int n_theta, double s_min, double s_max, int grid_mode, int vertex,
                   double cf, double D, double omega, double m, const double* A, const double* B,
                   const double* gA, const double* gB, double* gparams, double* lambda,
                   int nthreads) {
    const int nn = 2 * n;
    std::vector<double> J((size_t)nn * nn), dF((size_t)3 * nn);
    if (oracle_jacobian(n, n_theta, s_min, s_max, grid_mode, vertex, cf, D, omega, m, A, B,
                        J.data(), nthreads))
        return 1;
    if (oracle_param_jacobian(n, n_theta, s_min, s_max, grid_mode, vertex, cf, D, omega, m, A, B,
                              dF.data()))
        return 1;
    std::vector<double> M((size_t)nn * nn), lam(nn);
    for (int r = 0; r < nn; ++r)
        for (int cidx = 0; cidx < nn; ++cidx)
            M[(size_t)r * nn + cidx] = (r == cidx ? 1.0 : 0.0) - J[(size_t)cidx * nn + r];
    for (int i = 0; i < n; ++i) { lam[i] = gA[i]; lam[n + i] = gB[i]; }
    if (lu_solve(nn, M, lam.data())) return 1;
    for (int t = 0; t < 3; ++t) {
        double s = 0.0;
        for (int r = 0; r < nn; ++r) s += lam[r] * dF[(size_t)t * nn + r];
        gparams[t] = s;
    }
    gparams[3] = 0.0;
    if (lambda) for (int r = 0; r < nn; ++r) lambda[r] = lam[r];
    return 0;
}

/* Grid-truncated condensate  -<qbar q> = 4 N_c int d^4q/(2pi)^4 B/(q^2 A^2 + B^2)
 *                                      = N_c/(4 pi^2) sum_j W_j B_j/d_j      (N_c = 3). */
double oracle_condensate(int n, double s_min, double s_max, int grid_mode, const double* A,
                         const double* B) {
    Cfg c = make_cfg(n, 1, s_min, s_max, grid_mode, 0, 4.0 / 3.0);
    Grid g;
    if (build_grid(c, g)) return NAN;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double Aq = at_q<double>(c, g, A, j), Bq = at_q<double>(c, g, B, j);
        s += g.W[j] * Bq / (g.sq[j] * Aq * Aq + Bq * Bq);
    }
    return 3.0 / (4.0 * kPi * kPi) * s;
}

int oracle_num_threads_available(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
