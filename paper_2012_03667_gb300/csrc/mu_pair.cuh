// mu_pair.cuh -- the arithmetic of one (external, internal) pair of the quark gap equation at
// finite chemical potential mu, shared by the device kernels of k_mu.cu and a host test harness.
//
// Equation (the extension of Sec. II announced in Sec. V): S^-1(p~) = i g_vec.p_vec A
// + i g_4 p~_4 C + B with p~ = (p_vec, p_4 + i mu); the gluon momentum k = p - q stays real; the
// interaction is the Gaussian of Eq. IRGsQC times the Landau projector; the vertex is the
// Ball-Chiu construction from the Ward-Takahashi identity,
//   Gamma_nu = Sigma_nu g_nu + t_nu (g_vec.t_vec dA/2 + g_4 t_4 dC/2 - i dB),  t = q~ + p~,
//   Sigma = (A_q + A_p)/2 (spatial), (C_q + C_p)/2 (nu = 4),  dF = (F_q - F_p)/(q~^2 - p~^2).
// The projections A = tr[g_vec.p_vec S^-1]/(4 i p_vec^2), C = tr[g_4 S^-1]/(4 i p~_4) and
// B = tr[S^-1]/4 of the self-energy, worked out in closed form with p_vec along the third axis,
// make each pair's integrand c0 + c1 z + (d0 + d1 z)/k^2 in the cosine z between p_vec and q_vec,
// with complex c, d that depend on (|p_vec|, |q_vec|, p~_4, q~_4) but not on z.  So the angular
// integral needs four real moments per pair,
//   m0 = sum_k w_k e_k,  m1 = sum_k w_k e_k z_k,  n0 = sum_k w_k e_k / k^2,  n1 = sum_k w_k e_k z_k / k^2,
//   e_k = exp(-k^2/omega^2),  k^2 = (P - Q)^2 + h^2 + 2 P Q (1 - z_k),  h = p_4 - q_4,
// which do not depend on mu (p~_4 - q~_4 = h is real).  Five combinations of them cancel when
// formed from rounded moments; they are formed once in FP64 (mu_planes) and stored with the four
// moments.  The rest is per (pair, mu) complex arithmetic (mu_pair_add).
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define QMU_HD __host__ __device__ __forceinline__
#else
#define QMU_HD inline
#endif

namespace qmu {

constexpr int kPlanes = 9;            // stored real planes per pair
constexpr double kSkipExponent = 70;  // pairs with ((P-Q)^2 + h^2)/omega^2 above this are dropped

template <class T>
struct cx {
    T re, im;
};

template <class T> QMU_HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> QMU_HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> QMU_HD cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <class T> QMU_HD cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T> QMU_HD cx<T> operator*(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T> QMU_HD cx<T> operator*(T s, cx<T> a) { return {a.re * s, a.im * s}; }
template <class T> QMU_HD cx<T> cinv(cx<T> a) {
    const T s = T(1) / (a.re * a.re + a.im * a.im);
    return {a.re * s, -a.im * s};
}

// The nine stored planes of one pair from its raw FP64 moments; scale multiplies all of them (the
// internal point's weight times the constant part of the measure and interaction).
//   0 m0   1 m1   2 n0   3 n1
//   4 n0 - R n1                        R = Q/P
//   5 -2 Q^2 n0 + R (P^2 + Q^2) n1
//   6 m0 - h^2 n0
//   7 3 m0 - (P^2 + Q^2) n0 + 2 P Q n1
//   8 Q^2 n0 - P Q n1
// (m1 and n1 are non-negative: e_k / k^2 grows with z_k, and the nodes are symmetric.)
QMU_HD void mu_planes(double P, double Q, double h, double m0, double m1, double n0, double n1,
                      double scale, double* v) {
    const double R = Q / P, PP = P * P, QQ = Q * Q;
    v[0] = scale * m0;
    v[1] = scale * m1;
    v[2] = scale * n0;
    v[3] = scale * n1;
    v[4] = scale * (n0 - R * n1);
    v[5] = scale * (-2.0 * QQ * n0 + R * (PP + QQ) * n1);
    v[6] = scale * (m0 - h * h * n0);
    v[7] = scale * (3.0 * m0 - (PP + QQ) * n0 + 2.0 * P * Q * n1);
    v[8] = scale * (QQ * n0 - P * Q * n1);
}

// The raw moments of one pair over the angular rule (z_k, w_k), in FP64.
QMU_HD void mu_moments(double P, double Q, double h, double omega, int nz, const double* z,
                       const double* wz, double* m0, double* m1, double* n0, double* n1) {
    const double inv_w2 = 1.0 / (omega * omega);
    const double base = (P - Q) * (P - Q) + h * h, twoPQ = 2.0 * P * Q;
    double a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    for (int k = 0; k < nz; ++k) {
        const double k2 = base + twoPQ * (1.0 - z[k]);
        const double e = wz[k] * exp(-k2 * inv_w2);
        const double ek = e / k2;
        a0 += e;
        a1 += e * z[k];
        b0 += ek;
        b1 += ek * z[k];
    }
    *m0 = a0;
    *m1 = a1;
    *n0 = b0;
    *n1 = b1;
}

// Per-pair real combinations that involve no cancellation, formed from the stored planes.
template <class T>
struct PairReal {
    T h, pq2;                  // h = p_4 - q_4, (P - Q)(P + Q)
    T m0, n0, v4, v5, v6, v7, v8;
    T Mp, Np, Rm1, Rn1, kA, jA, b3, b4, b7, b9;
};

template <class T>
QMU_HD PairReal<T> mu_pair_real(const T* v, T P, T Q, T h) {
    PairReal<T> r;
    const T R = Q / P, PP = P * P, QQ = Q * Q, PQ = P * Q;
    r.h = h;
    r.pq2 = (P - Q) * (P + Q);
    r.m0 = v[0];
    r.n0 = v[2];
    r.v4 = v[4];
    r.v5 = v[5];
    r.v6 = v[6];
    r.v7 = v[7];
    r.v8 = v[8];
    const T m1 = v[1], n1 = v[3];
    r.Mp = v[0] + R * m1;
    r.Np = v[2] + R * n1;
    r.Rm1 = R * m1;
    r.Rn1 = R * n1;
    r.kA = -(QQ * v[0] + R * (PP + QQ) * T(0.5) * m1);
    r.jA = R * (PP - QQ) * T(0.5) * n1;
    r.b3 = (PP + QQ) * T(0.5) * v[0] + PQ * m1;
    r.b4 = (PP - QQ) * T(0.5) * v[2];
    r.b7 = -(QQ * v[0] + PQ * m1);
    r.b9 = QQ * v[2] + PQ * n1;
    return r;
}

// Propagator parts at an internal point: S(q~) = -i g_vec.q_vec sv - i g_4 q~_4 s4 + ss with
// (sv, s4, ss) = (A, C, B)/(q_vec^2 A^2 + q~_4^2 C^2 + B^2); returns s4q = s4 q~_4 in place of s4.
template <class T>
QMU_HD void mu_propagator(T Q, cx<T> qt, cx<T> A, cx<T> C, cx<T> B, cx<T>* sv, cx<T>* s4q,
                          cx<T>* ss) {
    const cx<T> d = (Q * Q) * (A * A) + (qt * qt) * (C * C) + B * B;
    const cx<T> id = cinv(d);
    *sv = A * id;
    *s4q = C * id * qt;
    *ss = B * id;
}

// Adds one pair's contribution at one mu: to SA (the A projection), SCp (the C projection times
// p~_4) and SB (the B projection).  s = p_4 + q_4 is real; p~_4 + q~_4 = s + 2 i mu.
// bc = false gives the bare vertex gamma_nu (rainbow truncation).
// (Adi, Cdi, Bdi): the values subtracted in the vertex's difference numerators F_q - F_p, which
// are the external point's own (Ai, Ci, Bi) except under reading M8 (k_mu.cu).
template <class T>
QMU_HD void mu_pair_add_dq(const PairReal<T>& r, T s, T mu, bool bc, cx<T> Ai, cx<T> Ci,
                           cx<T> Bi, cx<T> Adi, cx<T> Cdi, cx<T> Bdi, cx<T> Aj, cx<T> Cj,
                           cx<T> Bj, cx<T> sv, cx<T> s4q, cx<T> ss, cx<T>& SA, cx<T>& SCp,
                           cx<T>& SB) {
    const T h = r.h;
    if (!bc) {
        // Sigma = 1, no t-terms
        SA = SA + s4q * (T(2) * h * r.v4) + sv * (T(2) * r.Rm1 - h * h * r.Rn1 + r.v5);
        SB = SB + ss * (r.v6 + r.v7);
        SCp = SCp + s4q * (r.v7 - r.v6) + sv * (T(-2) * h * r.v8);
        return;
    }
    const cx<T> spl = {s, T(2) * mu};  // p~_4 + q~_4
    const cx<T> aA = (Aj + Ai) * T(0.5), aC = (Cj + Ci) * T(0.5), aAC = aA + aC;
    const cx<T> eA = Aj - Adi, eC = Cj - Cdi, eB = Bj - Bdi;
    const cx<T> w = {r.pq2 + h * s, T(2) * mu * h};  // p~^2 - q~^2
    const cx<T> iw = cinv(w);
    const cx<T> dA = -(eA * iw), dC = -(eC * iw), dB = -(eB * iw);  // (F_q - F_p)/(q~^2 - p~^2)
    const cx<T> hs = spl * T(0.5);                                  // (p~_4 + q~_4)/2
    const cx<T> spl2h = spl * hs;                                   // (p~_4 + q~_4)^2 / 2
    // A projection
    const cx<T> tA_ss = -(dB * r.Mp) - eB * r.v4;
    const cx<T> tA_s4 = -(hs * ((dC + dA) * r.Mp + eC * r.v4)) - eA * (T(0.5) * h * r.Np) +
                        aAC * (h * r.v4);
    const cx<T> tA_sv = aAC * r.Rm1 - aC * (h * h * r.Rn1) + aA * r.v5 + spl2h * dC * r.Rm1 +
                        hs * eC * (h * r.Rn1) + dA * r.kA - eA * r.jA;
    SA = SA + ss * tA_ss + s4q * tA_s4 + sv * tA_sv;
    // B and C projections share four structures
    const cx<T> T1 = -(spl * dB * r.m0) - eB * (h * r.n0);
    const cx<T> U = dA * r.b3 + eA * r.b4 + aA * r.v7;
    const cx<T> V = spl2h * dC * r.m0 + hs * eC * (h * r.n0) + aC * r.v6;
    SB = SB + ss * (U + V) + s4q * T1 + sv * (dB * r.b7 + eB * r.v8);
    const cx<T> tC_sv = hs * ((dC + dA) * r.b7 + eC * r.v8) - eA * (T(0.5) * h * r.b9) -
                        aAC * (h * r.v8);
    SCp = SCp + ss * T1 + s4q * (U - V) + sv * tC_sv;
}

template <class T>
QMU_HD void mu_pair_add(const PairReal<T>& r, T s, T mu, bool bc, cx<T> Ai, cx<T> Ci, cx<T> Bi,
                        cx<T> Aj, cx<T> Cj, cx<T> Bj, cx<T> sv, cx<T> s4q, cx<T> ss, cx<T>& SA,
                        cx<T>& SCp, cx<T>& SB) {
    mu_pair_add_dq<T>(r, s, mu, bc, Ai, Ci, Bi, Ai, Ci, Bi, Aj, Cj, Bj, sv, s4q, ss, SA, SCp, SB);
}

}  // namespace qmu
