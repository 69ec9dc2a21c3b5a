// f2.cuh -- double-float arithmetic on the FP32 pipe and the angular kernel entries of one pair
// evaluated with it; shared by the kernel precompute (k_precompute.cu) and a host test harness.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2 (48 significant bits,
// relative precision about 4e-15).  The building blocks are the error-free transformations of a
// sum (Knuth's TwoSum: a + b = s + e exactly for s = fl(a + b)) and of a product (with a fused
// multiply-add, a b = p + e exactly for p = fl(a b), e = fma(a, b, -p)); the operations on pairs
// combine them and renormalise.  Every step is written out explicitly (no expression the compiler
// could contract or reassociate changes an error term).
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define F2_HD __host__ __device__ __forceinline__
#else
#define F2_HD inline
#endif

namespace qf2 {

struct f2 {
    float h, l;
};

F2_HD float rn(double x) { return static_cast<float>(x); }  // round to nearest

F2_HD f2 of(double x) {
    const float h = rn(x);
    return {h, rn(x - static_cast<double>(h))};
}
F2_HD double val(f2 a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }
F2_HD f2 neg(f2 a) { return {-a.h, -a.l}; }

F2_HD f2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
F2_HD f2 fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
    const float s = a + b;
    return {s, b - (s - a)};
}
F2_HD f2 two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
F2_HD f2 mul(f2 a, f2 b) {
    f2 p = two_prod(a.h, b.h);
    p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
    return fast_two_sum(p.h, p.l);
}
// sum of two values of the same sign (no cancellation)
F2_HD f2 add_same(f2 a, f2 b) {
    f2 s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return fast_two_sum(s.h, s.l);
}
// sum of two values of any signs
F2_HD f2 add(f2 a, f2 b) {
    f2 s = two_sum(a.h, b.h);
    const f2 t = two_sum(a.l, b.l);
    s.l += t.h;
    s = fast_two_sum(s.h, s.l);
    s.l += t.l;
    return fast_two_sum(s.h, s.l);
}
F2_HD f2 div(f2 a, f2 b) {
    const float q1 = a.h / b.h;
    const f2 p = two_prod(q1, b.h);  // a.h - p.h is exact: p.h lies within a rounding of a.h
    const float r = fmaf(-q1, b.l, ((a.h - p.h) - p.l) + a.l);
    return fast_two_sum(q1, r / b.h);
}

// exp(-d) for a pair 0 <= d < kExpTop.  d = a/4 + b/512 + r with a = rint(4 d_h) and
// b = rint(512 (d_h - a/4)) in [-64, 64] (both subtractions exact by Sterbenz's lemma) and
// |r| <= 1/1024 + |d_l|; exp(-a/4) and exp(-b/512) come from tables of pairs (ta: a = 0 .. kExpA - 1,
// tb: b = -64 .. 64, each (h, l) interleaved) and exp(-r) from its Taylor polynomial
// 1 - r + r^2/2 - r^3/6 + r^4/24, whose next term is below 1e-17.
constexpr int kExpA = 352;
constexpr int kExpB = 129;
constexpr float kExpTop = 87.5f;  // exp(-87.5) ~ 1e-38: the FP32 range

// exp(-r) for |r| <= about 1/1024 (r a pair), times exp(-a/4) exp(-b/512) from the tables.
F2_HD f2 exp_neg_reduced(f2 r, int a, int b, const float* ta, const float* tb) {
    f2 r2 = two_prod(r.h, r.h);
    r2.l = fmaf(2.f * r.h, r.l, r2.l);
    const float tail = r.h * r2.h * fmaf(r.h, 1.f / 24.f, -1.f / 6.f);
    f2 e = two_sum(1.f, -r.h);
    const float el = ((e.l - r.l) + 0.5f * r2.l) + tail;
    const f2 q = two_sum(e.h, 0.5f * r2.h);
    e = fast_two_sum(q.h, q.l + el);
    const int ia = 2 * a, ib = 2 * (b + 64);
    return mul(mul({ta[ia], ta[ia + 1]}, {tb[ib], tb[ib + 1]}), e);
}

F2_HD f2 exp_neg(f2 d, const float* ta, const float* tb) {
    const float a = rintf(d.h * 4.f);
    const float u = fmaf(a, -0.25f, d.h);
    const float b = rintf(u * 512.f);
    const float rh = fmaf(b, -1.f / 512.f, u);
    return exp_neg_reduced(two_sum(rh, d.l), static_cast<int>(a), static_cast<int>(b), ta, tb);
}

// exp(-x) for an FP64 argument 0 <= x < kExpTop, reduced in FP64 (exactly) so that the argument
// keeps its full precision: a pair's factor exp(-ex_0) has ex_0 up to 87, where the 48-bit pair
// representation of the argument alone would cost up to 1e-13.
F2_HD f2 exp_neg_d(double x, const float* ta, const float* tb) {
    const double a = rint(x * 4.0);
    const double u = x - a * 0.25;
    const double b = rint(u * 512.0);
    return exp_neg_reduced(of(u - b * (1.0 / 512.0)), static_cast<int>(a), static_cast<int>(b),
                           ta, tb);
}

// Host: the tables of exp_neg from FP64 exp, kExpA + kExpB interleaved pairs.
inline void exp_tables(float* out) {
    for (int a = 0; a < kExpA; ++a) {
        const f2 v = of(std::exp(-0.25 * a));
        out[2 * a] = v.h;
        out[2 * a + 1] = v.l;
    }
    for (int b = -64; b <= 64; ++b) {
        const f2 v = of(std::exp(-b / 512.0));
        out[2 * (kExpA + b + 64)] = v.h;
        out[2 * (kExpA + b + 64) + 1] = v.l;
    }
}

// The angular kernels of one pair (P, Q) (Eqs. dsesys/dsesys2 after the traces; D factored out):
//   K_0 = pref S_0,  K_T = 2PQ pref S_t,  K_3 = 3 sqrt(PQ) pref S_z - K_T   (g_3 = 3x - g_T),
//   S_0 = sum_k w_k e_k,  S_z = sum_k w_k z_k e_k,  S_t = sum_k w_k (1 - z_k^2) e_k / k_k^2,
//   e_k = exp(-k_k^2/w^2),  k_k^2 = (sqrt P - sqrt Q)^2 + 2 sqrt(PQ) y_k,  y_k = 1 - z_k,
// with pref = 8 pi^2/w^4.  The exponent is split off the first node: k_k^2/w^2 = ex_0 + d_k,
// d_k = (2 sqrt(PQ)/w^2)(y_k - y_0) >= 0 increasing with k, so the sums carry exp(-d_k) and the
// factor pref exp(-ex_0) is applied once; the sum stops once d_k > cut (every later term is below
// e^-cut of the first times polynomial ratios).  Node tables (interleaved pairs): dy = y_k - y_0,
// w = w_k, wz = w_k z_k, ws = w_k (1 - z_k^2).  The pair constants are formed in FP64 from the FP64
// grid (dd = (sqrt P - sqrt Q)^2 keeps its full accuracy between neighbouring nodes).  Returns
// false, with zero entries, when ex_0 >= kExpTop: every term is then below the FP32 range.
F2_HD bool pair_entries(double P, double Q, double rP, double rQ, double y0, double iw2,
                        double pref, double cut, int nt, const float* dy, const float* w,
                        const float* wz, const float* ws, const float* ta, const float* tb,
                        f2& K0, f2& KT, f2& K3) {
    K0 = KT = K3 = {0.f, 0.f};
    const double dd = (rP - rQ) * (rP - rQ);
    const double c2 = 2.0 * rP * rQ;
    const double k20 = dd + c2 * y0;
    const double ex0 = k20 * iw2;
    if (!(ex0 < static_cast<double>(kExpTop))) return false;
    const f2 C2 = of(c2), Tw = of(c2 * iw2), K20 = of(k20);
    const float fcut = static_cast<float>(cut);
    // S_z is summed in two same-sign parts (z_k > 0, then z_k <= 0: the nodes run from z near 1
    // to z near -1) and the parts are subtracted once
    f2 S0 = {0.f, 0.f}, Szp = {0.f, 0.f}, Szn = {0.f, 0.f}, St = {0.f, 0.f};
    for (int k = 0; k < nt; ++k) {
        const f2 y = {dy[2 * k], dy[2 * k + 1]};
        const f2 d = mul(Tw, y);
        if (d.h > fcut) break;
        const f2 e = exp_neg(d, ta, tb);
        const f2 k2 = add_same(K20, mul(C2, y));
        S0 = add_same(S0, mul(e, {w[2 * k], w[2 * k + 1]}));
        const f2 ez = mul(e, {wz[2 * k], wz[2 * k + 1]});
        if (wz[2 * k] > 0.f) Szp = add_same(Szp, ez);
        else Szn = add_same(Szn, ez);
        St = add_same(St, div(mul(e, {ws[2 * k], ws[2 * k + 1]}), k2));
    }
    const f2 Sz = add(Szp, Szn);
    const f2 fac = mul(of(pref), exp_neg_d(ex0, ta, tb));
    K0 = mul(fac, S0);
    KT = mul(mul(fac, of(2.0 * P * Q)), St);
    K3 = add(mul(mul(fac, of(3.0 * rP * rQ)), Sz), neg(KT));
    return true;
}

}  // namespace qf2
