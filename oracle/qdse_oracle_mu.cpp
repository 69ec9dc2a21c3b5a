/*
 * qdse_oracle_mu.cpp -- plain, slow FP64 CPU oracle of one successive-approximation sweep of the
 * quark gap equation at finite quark chemical potential mu, with the Ball-Chiu-type vertex
 * (the extension announced in Sec. V of Huang, Duan, Hu, Chen, arXiv:2012.03667).
 *
 * TEST INFRASTRUCTURE ONLY.  Like qdse_oracle.cpp it is an independent checker: only the
 * test-suite may load it, and it shares no code with the CUDA path.  It computes every Dirac
 * structure by explicit 4x4 complex matrices (products, a numerical inverse, traces), so no
 * trace identity has to be derived by hand.
 *
 * The paper gives no equations for mu > 0.  Readings taken here:
 *   M1  S^-1(p~) = i g_vec.p_vec A + i g_4 p~_4 C + B, p~ = (p_vec, p_4 + i mu), with A, C, B
 *       complex functions of (|p_vec|, p_4).
 *   M2  the gap equation of Sec. II (Eq. gendse with the truncation of Eq. KernelAnsatz) with
 *       p -> p~ in the quark propagator and the vertex; the gluon momentum k = p - q stays real,
 *       the interaction is 8 pi^2 D/w^4 exp(-k^2/w^2) times the transverse projector (reading R2
 *       of the vacuum oracle), colour factor C_F (reading R5).
 *   M3  the vertex is the Ball-Chiu construction for M1 from the Ward-Takahashi identity
 *       i (q~ - p~)_mu Gamma_mu(q~, p~) = S^-1(q~) - S^-1(p~):
 *         Gamma_mu = Sigma_mu g_mu + t_mu (g_vec.t_vec Delta_A / 2 + g_4 t_4 Delta_C / 2 - i Delta_B)
 *       with Sigma_mu = (A_q + A_p)/2 for mu = 1, 2, 3 and (C_q + C_p)/2 for mu = 4, t = q~ + p~,
 *       Delta_F = (F_q - F_p)/(q~^2 - p~^2), q~^2 = q_vec^2 + q~_4^2 (complex, no conjugation).
 *       At mu = 0 with C = A it is the vacuum vertex (Eq. bcvtxmu, Eq. 2).
 *   M4  projections A = tr[g_vec.p_vec S^-1]/(4 i p_vec^2), C = tr[g_4 S^-1]/(4 i p~_4),
 *       B = tr[S^-1]/4, applied to S^-1(p~) = i g.p~ + m + Sigma(p~).
 *   M5  d^4q/(2 pi)^4 = 2 pi/(2 pi)^4 dq_4 |q|^2 d|q| dz, z the cosine between p_vec and q_vec:
 *       the projected traces are invariant under rotations about p_vec, so the azimuth gives 2 pi.
 *   M8  (optional, off by default) the difference numerators F_q - F_p of M3 may take, per pair,
 *       a caller-given value in place of F_p (oracle_mu_sweep_dq); the solve uses it for the
 *       ray-blended quotient of oracle_mu.py, which removes the runaway of the discrete
 *       principal-value sum at mu -> 0.
 * The quadrature (the internal points (|q|, q_4) with their weights, which include |q|^2, and the
 * z nodes and weights) is the caller's; the sweep is the plain sum over it.  Internal and
 * external points must differ (k^2 > 0): the removable point q~ = p~ is not treated here.
 */
#include <cmath>
#include <complex>
#include <cstring>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const double kPi = 3.141592653589793238462643383279502884;

struct M4 {  // a 4x4 complex matrix, row-major
    cd a[4][4];
};

M4 zero() {
    M4 r;
    for (auto& row : r.a)
        for (auto& x : row) x = 0.0;
    return r;
}

M4 mul(const M4& x, const M4& y) {
    M4 r = zero();
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < 4; ++j) r.a[i][j] += x.a[i][k] * y.a[k][j];
    return r;
}

void axpy(M4& r, cd s, const M4& x) {  // r += s x
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) r.a[i][j] += s * x.a[i][j];
}

cd trace(const M4& x) { return x.a[0][0] + x.a[1][1] + x.a[2][2] + x.a[3][3]; }

// Gauss-Jordan inverse with partial pivoting; false if singular.
bool inverse(const M4& x, M4& r) {
    cd w[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) w[i][j] = j < 4 ? x.a[i][j] : cd(i == j - 4 ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int i = c + 1; i < 4; ++i)
            if (std::abs(w[i][c]) > std::abs(w[piv][c])) piv = i;
        if (std::abs(w[piv][c]) == 0.0) return false;
        for (int j = 0; j < 8; ++j) std::swap(w[c][j], w[piv][j]);
        const cd inv = 1.0 / w[c][c];
        for (int j = 0; j < 8; ++j) w[c][j] *= inv;
        for (int i = 0; i < 4; ++i) {
            if (i == c) continue;
            const cd f = w[i][c];
            for (int j = 0; j < 8; ++j) w[i][j] -= f * w[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) r.a[i][j] = w[i][j + 4];
    return true;
}

// Euclidean hermitian Dirac matrices, {g_mu, g_nu} = 2 delta (chiral representation):
// g_k = [[0, -i sigma_k], [i sigma_k, 0]], g_4 = [[0, 1], [1, 0]]; index 0..2 = k, 3 = 4.
M4 gamma(int mu) {
    static const cd I(0.0, 1.0);
    const cd sig[3][2][2] = {{{0.0, 1.0}, {1.0, 0.0}},
                             {{0.0, -I}, {I, 0.0}},
                             {{1.0, 0.0}, {0.0, -1.0}}};
    M4 g = zero();
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            if (mu < 3) {
                g.a[i][2 + j] = -I * sig[mu][i][j];
                g.a[2 + i][j] = I * sig[mu][i][j];
            } else {
                g.a[i][2 + j] = (i == j) ? 1.0 : 0.0;
                g.a[2 + i][j] = (i == j) ? 1.0 : 0.0;
            }
        }
    return g;
}

struct Gammas {
    M4 g[4], one;
    Gammas() {
        for (int mu = 0; mu < 4; ++mu) g[mu] = gamma(mu);
        one = zero();
        for (int i = 0; i < 4; ++i) one.a[i][i] = 1.0;
    }
};

const Gammas& G() {
    static const Gammas g;
    return g;
}

// S^-1 at the complex 4-momentum v~ = (v[0..2], v4) (reading M1).
M4 sinv(const double* v, cd v4, cd A, cd C, cd B) {
    static const cd I(0.0, 1.0);
    M4 r = zero();
    for (int k = 0; k < 3; ++k) axpy(r, I * v[k] * A, G().g[k]);
    axpy(r, I * v4 * C, G().g[3]);
    axpy(r, B, G().one);
    return r;
}

// Gamma_nu(q~, p~) of reading M3 (vertex 0 = BC) or the bare g_nu (vertex 1 = rainbow).
// ApD, CpD, BpD: the values subtracted in the difference numerators (normally Ap, Cp, Bp).
void vertex(const double* q, cd q4, const double* p, cd p4, cd Aq, cd Cq, cd Bq, cd Ap, cd Cp,
            cd Bp, cd ApD, cd CpD, cd BpD, int rainbow, M4 out[4]) {
    static const cd I(0.0, 1.0);
    if (rainbow) {
        for (int nu = 0; nu < 4; ++nu) out[nu] = G().g[nu];
        return;
    }
    const cd t[4] = {q[0] + p[0], q[1] + p[1], q[2] + p[2], q4 + p4};
    const cd q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q4 * q4;
    const cd p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + p4 * p4;
    const cd den = q2 - p2;
    const cd dA = (Aq - ApD) / den, dC = (Cq - CpD) / den, dB = (Bq - BpD) / den;
    // the t-structure: g_vec.t_vec dA/2 + g_4 t_4 dC/2 - i dB
    M4 X = zero();
    for (int k = 0; k < 3; ++k) axpy(X, 0.5 * t[k] * dA, G().g[k]);
    axpy(X, 0.5 * t[3] * dC, G().g[3]);
    axpy(X, -I * dB, G().one);
    for (int nu = 0; nu < 4; ++nu) {
        out[nu] = zero();
        axpy(out[nu], nu < 3 ? 0.5 * (Aq + Ap) : 0.5 * (Cq + Cp), G().g[nu]);
        axpy(out[nu], t[nu], X);
    }
}

}  // namespace

extern "C" {

// The vertex and the inverse propagators at (q~, p~), for the Ward-Takahashi check.  Complex
// values interleaved (re, im); matrices row-major: gam[4][16], sq[16], sp[16].
void oracle_mu_vertex(const double* q, double q4r, double q4i, const double* p, double p4r,
                      double p4i, const double* qf /*Aq, Cq, Bq*/, const double* pf /*Ap, Cp, Bp*/,
                      int rainbow, double* gam, double* sq, double* sp) {
    const cd q4(q4r, q4i), p4(p4r, p4i);
    const cd Aq(qf[0], qf[1]), Cq(qf[2], qf[3]), Bq(qf[4], qf[5]);
    const cd Ap(pf[0], pf[1]), Cp(pf[2], pf[3]), Bp(pf[4], pf[5]);
    M4 g[4];
    vertex(q, q4, p, p4, Aq, Cq, Bq, Ap, Cp, Bp, Ap, Cp, Bp, rainbow, g);
    const M4 Sq = sinv(q, q4, Aq, Cq, Bq), Sp = sinv(p, p4, Ap, Cp, Bp);
    for (int nu = 0; nu < 4; ++nu)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                gam[2 * (16 * nu + 4 * i + j)] = g[nu].a[i][j].real();
                gam[2 * (16 * nu + 4 * i + j) + 1] = g[nu].a[i][j].imag();
            }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            sq[2 * (4 * i + j)] = Sq.a[i][j].real();
            sq[2 * (4 * i + j) + 1] = Sq.a[i][j].imag();
            sp[2 * (4 * i + j)] = Sp.a[i][j].real();
            sp[2 * (4 * i + j) + 1] = Sp.a[i][j].imag();
        }
}

// One sweep (readings M1-M5): for every external point i (|p_vec| = pv[i], p_4 = p4[i]) the new
// A, C, B from the inputs at the external points (Ap, Cp, Bp, used in the vertex) and at the
// internal points j (|q_vec| = qv[j], q_4 = q4[j], weight wq[j] for dq_4 |q|^2 d|q|), with nz
// cosine nodes z (weights wz).  Complex arrays interleaved (re, im).  Fd (M8): NULL, or complex
// [3][np * nq] -- per pair (i, j), the A, C, B subtracted in the difference numerators in place
// of Ap[i], Cp[i], Bp[i].  Returns 0, or 1 when a propagator is singular or k^2 = 0 at some point.
int oracle_mu_sweep_dq(int np, const double* pv, const double* p4, int nq, const double* qv,
                       const double* q4, const double* wq, int nz, const double* z,
                       const double* wz, double D, double omega, double m, double mu, double cf,
                       int rainbow, const double* Ap, const double* Cp, const double* Bp,
                       const double* Aq, const double* Cq, const double* Bq, const double* Fd,
                       double* Ao, double* Co, double* Bo, int nthreads) {
    static const cd I(0.0, 1.0);
    const double pref = cf * 8.0 * kPi * kPi * D / (omega * omega * omega * omega);
    const double measure = 2.0 * kPi / std::pow(2.0 * kPi, 4);
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
#endif
    for (int i = 0; i < np; ++i) {
        const double p[3] = {0.0, 0.0, pv[i]};  // p_vec along the third axis
        const cd pt4(p4[i], mu);
        const cd Api(Ap[2 * i], Ap[2 * i + 1]), Cpi(Cp[2 * i], Cp[2 * i + 1]),
            Bpi(Bp[2 * i], Bp[2 * i + 1]);
        cd sa = 0.0, sc = 0.0, sb = 0.0;
        for (int j = 0; j < nq; ++j) {
            const cd qt4(q4[j], mu);
            const cd Aqj(Aq[2 * j], Aq[2 * j + 1]), Cqj(Cq[2 * j], Cq[2 * j + 1]),
                Bqj(Bq[2 * j], Bq[2 * j + 1]);
            for (int k = 0; k < nz; ++k) {
                const double sn = std::sqrt(std::fmax(0.0, 1.0 - z[k] * z[k]));
                const double q[3] = {qv[j] * sn, 0.0, qv[j] * z[k]};
                const double kv[4] = {p[0] - q[0], p[1] - q[1], p[2] - q[2], p4[i] - q4[j]};
                const double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2] + kv[3] * kv[3];
                if (!(k2 > 0.0)) {
                    bad = 1;
                    continue;
                }
                M4 S;
                if (!inverse(sinv(q, qt4, Aqj, Cqj, Bqj), S)) {
                    bad = 1;
                    continue;
                }
                cd AD = Api, CD = Cpi, BD = Bpi;
                if (Fd) {
                    const size_t o = (size_t)i * nq + j, npq = (size_t)np * nq;
                    AD = cd(Fd[2 * o], Fd[2 * o + 1]);
                    CD = cd(Fd[2 * (npq + o)], Fd[2 * (npq + o) + 1]);
                    BD = cd(Fd[2 * (2 * npq + o)], Fd[2 * (2 * npq + o) + 1]);
                }
                M4 Gam[4];
                vertex(q, qt4, p, pt4, Aqj, Cqj, Bqj, Api, Cpi, Bpi, AD, CD, BD, rainbow, Gam);
                // sum_{mu nu} T_mu nu(k) g_mu S Gamma_nu, T = delta - k k / k^2
                M4 Msum = zero();
                for (int a = 0; a < 4; ++a) {
                    M4 Ta = zero();
                    for (int b = 0; b < 4; ++b)
                        axpy(Ta, (a == b ? 1.0 : 0.0) - kv[a] * kv[b] / k2, Gam[b]);
                    const M4 t = mul(G().g[a], mul(S, Ta));
                    axpy(Msum, 1.0, t);
                }
                const double wgt = measure * wq[j] * wz[k] * pref * std::exp(-k2 / (omega * omega));
                sa += wgt * trace(mul(G().g[2], Msum)) / (4.0 * I * pv[i]);
                sc += wgt * trace(mul(G().g[3], Msum)) / (4.0 * I * pt4);
                sb += wgt * trace(Msum) / 4.0;
            }
        }
        const cd A1 = 1.0 + sa, C1 = 1.0 + sc, B1 = m + sb;
        Ao[2 * i] = A1.real();
        Ao[2 * i + 1] = A1.imag();
        Co[2 * i] = C1.real();
        Co[2 * i + 1] = C1.imag();
        Bo[2 * i] = B1.real();
        Bo[2 * i + 1] = B1.imag();
    }
    return bad;
}

// oracle_mu_sweep_dq without M8: the exact difference numerators of M3.
int oracle_mu_sweep(int np, const double* pv, const double* p4, int nq, const double* qv,
                    const double* q4, const double* wq, int nz, const double* z,
                    const double* wz, double D, double omega, double m, double mu, double cf,
                    int rainbow, const double* Ap, const double* Cp, const double* Bp,
                    const double* Aq, const double* Cq, const double* Bq, double* Ao, double* Co,
                    double* Bo, int nthreads) {
    return oracle_mu_sweep_dq(np, pv, p4, nq, qv, q4, wq, nz, z, wz, D, omega, m, mu, cf, rainbow,
                              Ap, Cp, Bp, Aq, Cq, Bq, nullptr, Ao, Co, Bo, nthreads);
}

}  // extern "C"
