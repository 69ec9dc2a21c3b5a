// Host harness (test-suite only): the double-float arithmetic of the kernel precompute
// (paper_2012_03667_gb300/csrc/f2.cuh) compiled with the host compiler, so the test can compare the
// per-pair kernel entries the GPU stores with extended-precision sums of their definition.
#include <vector>

#include "../../paper_2012_03667_gb300/csrc/f2.cuh"

namespace {
std::vector<float> g_tab;
const float* tables() {
    if (g_tab.empty()) {
        g_tab.resize(2 * (qf2::kExpA + qf2::kExpB));
        qf2::exp_tables(g_tab.data());
    }
    return g_tab.data();
}
}  // namespace

extern "C" {

// exp(-d) of a pair d = (dh, dl): out = h + l
double host_exp_neg(float dh, float dl) {
    const float* t = tables();
    return qf2::val(qf2::exp_neg({dh, dl}, t, t + 2 * qf2::kExpA));
}

// The entries K_0, K_T (not divided by Q - P), K_3 of one pair as the precompute forms them, from
// the FP64 angular rule (y = 1 - z, z, s2 = 1 - z^2, w): out[3].  Returns 0 when the pair is stored
// as zeros (its first term is below the FP32 range).
int host_pair_entries(double P, double Q, double omega, int nt, const double* y, const double* z,
                      const double* s2, const double* w, double cut, double* out) {
    std::vector<float> dy(2 * nt), ww(2 * nt), wz(2 * nt), ws(2 * nt);
    for (int k = 0; k < nt; ++k) {
        const qf2::f2 a = qf2::of(y[k] - y[0]), b = qf2::of(w[k]), c = qf2::of(w[k] * z[k]),
                      d = qf2::of(w[k] * s2[k]);
        dy[2 * k] = a.h; dy[2 * k + 1] = a.l;
        ww[2 * k] = b.h; ww[2 * k + 1] = b.l;
        wz[2 * k] = c.h; wz[2 * k + 1] = c.l;
        ws[2 * k] = d.h; ws[2 * k + 1] = d.l;
    }
    const double pi = 3.141592653589793238462643383279502884;
    const double iw2 = 1.0 / (omega * omega);
    const double pref = 8.0 * pi * pi / (omega * omega * omega * omega);
    const float* t = tables();
    qf2::f2 K0, KT, K3;
    const bool kept = qf2::pair_entries(P, Q, std::sqrt(P), std::sqrt(Q), y[0], iw2, pref, cut, nt,
                                        dy.data(), ww.data(), wz.data(), ws.data(), t,
                                        t + 2 * qf2::kExpA, K0, KT, K3);
    out[0] = qf2::val(K0);
    out[1] = qf2::val(KT);
    out[2] = qf2::val(K3);
    return kept ? 1 : 0;
}

}  // extern "C"
