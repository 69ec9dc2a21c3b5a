// Host harness (test-suite only): one finite-mu sweep from the pair arithmetic the CUDA kernels
// use (paper_2012_03667_gb300/csrc/mu_pair.cuh), as plain loops over every (external, internal)
// pair, in FP64 or FP32, without the kernels' windows.  The test compares it with the FP64 oracle.
#include <complex>
#include <vector>

#include "../../paper_2012_03667_gb300/csrc/mu_pair.cuh"

namespace {

template <class T>
void sweep(int np, const double* pv, const double* p4, int nq, const double* qv, const double* q4,
           const double* wq, int nz, const double* z, const double* wz, double D, double omega,
           double m, double mu, double cf, int rainbow, const double* Fp, const double* Fq,
           double* Fo) {
    using C = qmu::cx<T>;
    auto ld = [](const double* a, int i) { return C{T(a[2 * i]), T(a[2 * i + 1])}; };
    const double kPi = 3.141592653589793238462643383279502884;
    const double kappa = cf * D / (kPi * omega * omega * omega * omega);
    for (int i = 0; i < np; ++i) {
        const C Ai = ld(Fp, i), Ci = ld(Fp + 2 * np, i), Bi = ld(Fp + 4 * np, i);
        C SA{0, 0}, SC{0, 0}, SB{0, 0};
        for (int j = 0; j < nq; ++j) {
            double m0, m1, n0, n1, v[qmu::kPlanes];
            const double h = p4[i] - q4[j];
            qmu::mu_moments(pv[i], qv[j], h, omega, nz, z, wz, &m0, &m1, &n0, &n1);
            qmu::mu_planes(pv[i], qv[j], h, m0, m1, n0, n1, wq[j], v);
            T vt[qmu::kPlanes];
            for (int c = 0; c < qmu::kPlanes; ++c) vt[c] = T(v[c]);
            const qmu::PairReal<T> r = qmu::mu_pair_real<T>(vt, T(pv[i]), T(qv[j]), T(h));
            // propagator parts formed in FP64, then rounded (as the prep kernel does)
            qmu::cx<double> sv, s4q, ss;
            const qmu::cx<double> qt{q4[j], mu};
            qmu::mu_propagator<double>(qv[j], qt, {Fq[2 * j], Fq[2 * j + 1]},
                                       {Fq[2 * nq + 2 * j], Fq[2 * nq + 2 * j + 1]},
                                       {Fq[4 * nq + 2 * j], Fq[4 * nq + 2 * j + 1]}, &sv, &s4q, &ss);
            qmu::mu_pair_add<T>(r, T(p4[i] + q4[j]), T(mu), !rainbow, Ai, Ci, Bi, ld(Fq, j),
                                ld(Fq + 2 * nq, j), ld(Fq + 4 * nq, j), C{T(sv.re), T(sv.im)},
                                C{T(s4q.re), T(s4q.im)}, C{T(ss.re), T(ss.im)}, SA, SC, SB);
        }
        const std::complex<double> pt(p4[i], mu);
        const std::complex<double> a = 1.0 + kappa * std::complex<double>(SA.re, SA.im);
        const std::complex<double> c = 1.0 + kappa * std::complex<double>(SC.re, SC.im) / pt;
        const std::complex<double> b = m + kappa * std::complex<double>(SB.re, SB.im);
        Fo[2 * i] = a.real(); Fo[2 * i + 1] = a.imag();
        Fo[2 * np + 2 * i] = c.real(); Fo[2 * np + 2 * i + 1] = c.imag();
        Fo[4 * np + 2 * i] = b.real(); Fo[4 * np + 2 * i + 1] = b.imag();
    }
}

}  // namespace

// F arrays: complex interleaved, [3][n] (A, C, B).  fp32 != 0 runs the pair arithmetic in FP32.
extern "C" void host_mu_sweep(int np, const double* pv, const double* p4, int nq, const double* qv,
                              const double* q4, const double* wq, int nz, const double* z,
                              const double* wz, double D, double omega, double m, double mu,
                              double cf, int rainbow, int fp32, const double* Fp, const double* Fq,
                              double* Fo) {
    if (fp32)
        sweep<float>(np, pv, p4, nq, qv, q4, wq, nz, z, wz, D, omega, m, mu, cf, rainbow, Fp, Fq, Fo);
    else
        sweep<double>(np, pv, p4, nq, qv, q4, wq, nz, z, wz, D, omega, m, mu, cf, rainbow, Fp, Fq,
                      Fo);
}
