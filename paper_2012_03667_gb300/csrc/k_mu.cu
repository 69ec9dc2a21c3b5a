// k_mu.cu -- finite chemical potential: the angular-moment table, the propagator prep and the
// batched sweep (include/qdse_mu.h), for sm_103a.
//
// The sweep of the gap equation at finite mu (Sec. V extension of Sec. II) is, per external point
// p and chemical potential mu, a sum over internal points q of complex structures built from
// A, C, B at p and q, times four real angular moments of the Gaussian interaction (mu_pair.cuh).
// The moments do not depend on mu, so they are formed once per (omega, grid) in FP64 and stored;
// every sweep of every mu reads them.  Layout in HBM:
//   table  T[9 * n_pairs]: external point e owns pairs [off_e, off_e + len_e); its internal points
//          are a window r in [r_lo, r_lo + nr_e) x f in [f_lo, f_lo + nf_e) of the product grid
//          (the rest are below exp(-70)); plane c of e is the contiguous run
//          table[9 off_e + c len_e + jj], jj = (r - r_lo) nf_e + (f - f_lo), so that consecutive
//          threads read consecutive words of every plane.
//   vec    T[n_mu][n_int][12]: A, C, B, sv, s4 q~_4, ss at each internal point for each mu
//          ((re, im) pairs; 48 B per point in FP32, read as three 16-byte loads), written by
//          k_mu_prep once per sweep.
// k_mu_sweep gives each warp one (external point, tile of TB chemical potentials): its lanes take
// pairs jj = lane, lane + 32, ...; each lane loads a pair's 9 planes once and applies them to the
// TB chemical potentials of the tile (the table is read n_mu/TB times per sweep), and the warp
// reduces its sums with shuffles (no block barrier).  Consecutive warps take consecutive external
// points of the same tile, so the tile's vectors stay in L2 while the table streams from HBM.
// The tile's values at the external point sit in shared memory, which keeps the FP32 kernel at
// 128 registers (4 blocks of 4 warps per SM).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/qdse.h"
#include "../../include/qdse_mu.h"
#include "mu_pair.cuh"

namespace {

thread_local std::string g_mu_err;

int mu_fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_mu_err = buf;
    return status;
}

int mu_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return QDSE_OK;
    return mu_fail(e == cudaErrorMemoryAllocation ? QDSE_ERR_OOM : QDSE_ERR_CUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

struct MuRow {
    long long off;     // first pair of this external point
    int len;           // pairs kept: nr * nf
    int r_lo, f_lo;    // window origin in the product grid
    int nf;            // window width in f (>= 1)
    double P, p4;      // |p_vec|, p_4
};

constexpr int kSweepThreads = 128;  // 4 independent warps per block
constexpr int kMomentThreads = 256;
constexpr int kTileF32 = 8;  // chemical potentials per warp, FP32 sweep
constexpr int kTileF64 = 4;  // chemical potentials per warp, FP64 sweep
constexpr int kMaxZ = 1024;
constexpr double kPi = 3.141592653589793238462643383279502884;

// ---- the moment table ------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kMomentThreads)
k_mu_moments(const MuRow* __restrict__ rows, const double* __restrict__ qr,
             const double* __restrict__ q4, const double* __restrict__ wq, int n_4, int nz,
             const double* __restrict__ z_g, const double* __restrict__ wz_g, double omega,
             double scale, T* __restrict__ table) {
    extern __shared__ double zs[];  // z[nz], wz[nz]
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        zs[k] = z_g[k];
        zs[nz + k] = wz_g[k];
    }
    __syncthreads();
    const MuRow row = rows[blockIdx.x];
    T* base = table + 9 * row.off;
    for (int jj = threadIdx.x; jj < row.len; jj += blockDim.x) {
        const int r = row.r_lo + jj / row.nf, f = row.f_lo + jj % row.nf;
        const double Q = qr[r], h = row.p4 - q4[f];
        double m0, m1, n0, n1, v[qmu::kPlanes];
        qmu::mu_moments(row.P, Q, h, omega, nz, zs, zs + nz, &m0, &m1, &n0, &n1);
        qmu::mu_planes(row.P, Q, h, m0, m1, n0, n1, scale * wq[(size_t)r * n_4 + f], v);
#pragma unroll
        for (int c = 0; c < qmu::kPlanes; ++c) base[(size_t)c * row.len + jj] = T(v[c]);
    }
}

// ---- per (mu, internal point): the propagator parts --------------------------------------------
template <class T>
__global__ void k_mu_prep(int n_mu, const double* __restrict__ mu, int n_int, int n_4,
                          const double* __restrict__ qr, const double* __restrict__ q4,
                          const double* __restrict__ F_int, T* __restrict__ vec) {
    using C = qmu::cx<double>;
    const size_t total = (size_t)n_mu * n_int;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / n_int), j = (int)(t % n_int);
        const int r = j / n_4, f = j % n_4;
        const double* Fb = F_int + (size_t)b * 6 * n_int;  // [3][n_int] complex
        const C A{Fb[2 * j], Fb[2 * j + 1]};
        const C Cc{Fb[2 * n_int + 2 * j], Fb[2 * n_int + 2 * j + 1]};
        const C B{Fb[4 * n_int + 2 * j], Fb[4 * n_int + 2 * j + 1]};
        C sv, s4q, ss;
        qmu::mu_propagator<double>(qr[r], C{q4[f], mu[b]}, A, Cc, B, &sv, &s4q, &ss);
        const double vals[12] = {A.re, A.im, Cc.re, Cc.im, B.re, B.im,
                                 sv.re, sv.im, s4q.re, s4q.im, ss.re, ss.im};
        T* vb = vec + t * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) vb[c] = T(vals[c]);
    }
}

// Reading M6 for one internal point: the four external corners (|p| lower/upper x p_4
// lower/upper, flat indices i * n_p4 + k), the weights of the upper |p| node (a) and of the upper
// p_4 node (b), and whether the point mirrors q_4 < 0 (value conjugated).
struct MuInterp {
    int e00, e10, e01, e11;
    double a, b;
    int conj, pad;
};

// Propagator parts of one (mu, internal point) from its A, C, B; stored as 12 values in T.
template <class T>
__device__ __forceinline__ void prep_store(qmu::cx<double> A, qmu::cx<double> Cc,
                                           qmu::cx<double> B, double Q, double q4f, double mu_b,
                                           T* vb) {
    qmu::cx<double> sv, s4q, ss;
    qmu::mu_propagator<double>(Q, qmu::cx<double>{q4f, mu_b}, A, Cc, B, &sv, &s4q, &ss);
    const double vals[12] = {A.re, A.im, Cc.re, Cc.im, B.re, B.im,
                             sv.re, sv.im, s4q.re, s4q.im, ss.re, ss.im};
#pragma unroll
    for (int c = 0; c < 12; ++c) vb[c] = T(vals[c]);
}

// As k_mu_prep, with A, C, B at the internal points interpolated from the external values.
// list: NULL, or the chemical potentials to prepare (compact slot cb holds list[cb]); vec is
// indexed by slot.
template <class T>
__global__ void k_mu_prep_interp(int n_act, const int* __restrict__ list,
                                 const double* __restrict__ mu, int n_int, int n_4,
                                 const double* __restrict__ qr, const double* __restrict__ q4,
                                 const MuInterp* __restrict__ interp,
                                 const double* __restrict__ F_ext, int n_ext, T* __restrict__ vec) {
    using C = qmu::cx<double>;
    const size_t total = (size_t)n_act * n_int;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int cb = (int)(t / n_int), j = (int)(t % n_int);
        const int b = list ? list[cb] : cb;
        const MuInterp ip = interp[j];
        const double w00 = (1.0 - ip.a) * (1.0 - ip.b), w10 = ip.a * (1.0 - ip.b);
        const double w01 = (1.0 - ip.a) * ip.b, w11 = ip.a * ip.b;
        C v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double* Fc = F_ext + ((size_t)b * 3 + c) * 2 * n_ext;
            C x = C{Fc[2 * ip.e00], Fc[2 * ip.e00 + 1]} * w00 +
                  C{Fc[2 * ip.e10], Fc[2 * ip.e10 + 1]} * w10;
            x = x + C{Fc[2 * ip.e01], Fc[2 * ip.e01 + 1]} * w01;
            x = x + C{Fc[2 * ip.e11], Fc[2 * ip.e11 + 1]} * w11;
            if (ip.conj) x.im = -x.im;
            v[c] = x;
        }
        prep_store<T>(v[0], v[1], v[2], qr[j / n_4], q4[j % n_4], mu[b], vec + t * 12);
    }
}

// One relaxation step and the convergence measure of reading M7, one block per chemical
// potential: F <- G (alpha = 1) or (1 - alpha) F + alpha G; change[b] = max over A, C, B of
// max|F_new - F_old| / max|F_new| (absolute where max|F_new| = 0); bad[b] = non-finite value.
// Chemical potentials with done[b] set are left as they are.
constexpr int kRelaxThreads = 256;
__global__ void __launch_bounds__(kRelaxThreads)
k_mu_relax(int n_ext, double alpha, double* __restrict__ F, const double* __restrict__ G,
           const int* __restrict__ done, double* __restrict__ change, int* __restrict__ bad) {
    const int b = blockIdx.x;
    if (done[b]) return;  // uniform over the block
    double md[3] = {0, 0, 0}, mm[3] = {0, 0, 0};
    int nonfinite = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double* Fc = F + ((size_t)b * 3 + c) * 2 * n_ext;
        const double* Gc = G + ((size_t)b * 3 + c) * 2 * n_ext;
        for (int e = threadIdx.x; e < n_ext; e += blockDim.x) {
            const double fr = Fc[2 * e], fi = Fc[2 * e + 1];
            double nr = Gc[2 * e], ni = Gc[2 * e + 1];
            if (alpha != 1.0) {
                nr = (1.0 - alpha) * fr + alpha * nr;
                ni = (1.0 - alpha) * fi + alpha * ni;
            }
            if (!isfinite(nr) || !isfinite(ni)) nonfinite = 1;
            md[c] = fmax(md[c], hypot(nr - fr, ni - fi));
            mm[c] = fmax(mm[c], hypot(nr, ni));
            Fc[2 * e] = nr;
            Fc[2 * e + 1] = ni;
        }
    }
    __shared__ double red[kRelaxThreads / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double x[6] = {md[0], md[1], md[2], mm[0], mm[1], mm[2]};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[k] = fmax(x[k], __shfl_down_sync(0xffffffffu, x[k], o));
        if (lane == 0) red[warp][k] = x[k];
    }
    const int any_bad = __syncthreads_or(nonfinite);
    if (threadIdx.x == 0) {
        double ch = 0;
        for (int c = 0; c < 3; ++c) {
            double d = 0, m = 0;
            for (int w = 0; w < kRelaxThreads / 32; ++w) {
                d = fmax(d, red[w][c]);
                m = fmax(m, red[w][3 + c]);
            }
            ch = fmax(ch, m > 0 ? d / m : d);
        }
        change[b] = ch;
        bad[b] = any_bad;
    }
}

// ---- the sweep ------------------------------------------------------------------------------------
// The 12 values of one (mu, internal point): three 16-byte loads in FP32, six in FP64.
template <class T>
__device__ __forceinline__ void load_point(const T* p, qmu::cx<T>* x);
template <>
__device__ __forceinline__ void load_point<float>(const float* p, qmu::cx<float>* x) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = q[0], b = q[1], c = q[2];
    x[0] = {a.x, a.y}; x[1] = {a.z, a.w}; x[2] = {b.x, b.y};
    x[3] = {b.z, b.w}; x[4] = {c.x, c.y}; x[5] = {c.z, c.w};
}
template <>
__device__ __forceinline__ void load_point<double>(const double* p, qmu::cx<double>* x) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double2 v = q[k];
        x[k] = {v.x, v.y};
    }
}

// Reading M8 (optional): the difference numerators F_q - F_p of the vertex take, per pair,
// F_p + beta (F_ray - F_p) in place of F_p, with F_ray the interpolation (reading M6) of F where q~'s
// ray crosses p~'s real 4-radius, (|q|, q_4) sqrt(P^2 + p_4^2)/sqrt(Q^2 + q_4^2), and
// beta = exp(-(2 mu |q_4 - p_4|/eta)^2).  The ray point depends on the pair only; beta on the
// pair and mu.  Pairs with beta below exp(-39.2) keep F_p (the difference is below 1e-17 of F).
struct RayArgs {
    const double* pax;   // external product grid: |p| axis [n_pr]
    const double* p4ax;  // p_4 axis [n_p4]
    int n_pr, n_p4;
    double eta;          // GeV^2
};
constexpr float kRayCut = 39.2f;  // beta = exp(-u^2) is kept while u^2 < 39.2

// (lower index, upper index, weight of the upper node) of x on an ascending axis: held at the first
// or last node outside it (the rule of reading M6, as in bracket() on the host).  In the sweep's
// precision T: FP32 sweeps only bring an FP32-accurate iterate to the FP64 phase.
template <class T>
__device__ __forceinline__ void ray_bracket(const double* __restrict__ axis, int n, T x, int& i0,
                                            int& i1, T& wgt) {
    int lo = -1, hi = n;  // axis[lo] <= x < axis[hi] (lo = -1: below the first node)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (T(axis[mid]) <= x) lo = mid;
        else hi = mid;
    }
    if (lo < 0) {
        i0 = i1 = 0;
        wgt = T(0);
    } else if (lo >= n - 1) {
        i0 = i1 = n - 1;
        wgt = T(0);
    } else {
        i0 = lo;
        i1 = lo + 1;
        wgt = (x - T(axis[lo])) / (T(axis[lo + 1]) - T(axis[lo]));
    }
}

template <class T, int TB, int MINB, bool RAY>
__global__ void __launch_bounds__(kSweepThreads, MINB)
k_mu_sweep(const MuRow* __restrict__ rows, const double* __restrict__ qr,
           const double* __restrict__ q4, const T* __restrict__ table, const T* __restrict__ vec,
           int n_int, int n_4, int n_mu, const int* __restrict__ list, int n_tiles,
           const double* __restrict__ mu, const double* __restrict__ F_ext, int n_ext,
           double kappa, double m_cur, int bc, double* __restrict__ F_out, RayArgs ray) {
    // n_mu slots; slot cb is chemical potential list[cb] (cb itself when list is NULL): F_ext,
    // F_out and mu are indexed by the chemical potential, vec by the slot.
    using C = qmu::cx<T>;
    constexpr int kW = kSweepThreads / 32;
    __shared__ T ext[kW][TB][7];  // A, C, B at the external point and mu, per slot of the tile
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * kW + wib;
    if (item >= (long long)n_ext * n_tiles) return;  // whole warps only; no block barrier below
    const int e = (int)(item % n_ext), b0 = (int)(item / n_ext) * TB;
    const int nb = min(TB, n_mu - b0);
    const MuRow row = rows[e];
    if (lane < TB) {
        const int cb = b0 + (lane < nb ? lane : 0);
        const int b = list ? list[cb] : cb;
        const double* Fb = F_ext + (size_t)b * 6 * n_ext;
        T* d = ext[wib][lane];
        d[0] = T(Fb[2 * e]);
        d[1] = T(Fb[2 * e + 1]);
        d[2] = T(Fb[2 * n_ext + 2 * e]);
        d[3] = T(Fb[2 * n_ext + 2 * e + 1]);
        d[4] = T(Fb[4 * n_ext + 2 * e]);
        d[5] = T(Fb[4 * n_ext + 2 * e + 1]);
        d[6] = T(mu[b]);
    }
    __syncwarp();
    const T P = T(row.P);
    C SA[TB], SC[TB], SB[TB];
#pragma unroll
    for (int t = 0; t < TB; ++t) SA[t] = SC[t] = SB[t] = C{T(0), T(0)};
    const T* base = table + 9 * row.off;
    for (int jj = lane; jj < row.len; jj += 32) {
        const int r = row.r_lo + jj / row.nf, f = row.f_lo + jj % row.nf;
        const int j = r * n_4 + f;
        T v[qmu::kPlanes];
#pragma unroll
        for (int c = 0; c < qmu::kPlanes; ++c) v[c] = base[(size_t)c * row.len + jj];
        const double q4f = q4[f];
        const qmu::PairReal<T> pr = qmu::mu_pair_real<T>(v, P, T(qr[r]), T(row.p4 - q4f));
        const T s = T(row.p4 + q4f);
        // reading M8: the ray point's corners and weights (reading M6), once per pair
        int e00 = 0, e10 = 0, e01 = 0, e11 = 0, rconj = 0;
        T ra = T(0), rb = T(0), dq4 = T(0);
        if (RAY) {
            const T Q = T(qr[r]), Pp = T(row.P), p4 = T(row.p4), q4 = T(q4f);
            const T lam = sqrt(Pp * Pp + p4 * p4) / sqrt(Q * Q + q4 * q4);
            int i0, i1, k0, k1;
            ray_bracket<T>(ray.pax, ray.n_pr, Q * lam, i0, i1, ra);
            ray_bracket<T>(ray.p4ax, ray.n_p4, fabs(q4 * lam), k0, k1, rb);
            dq4 = T(2) * T(fabs(row.p4 - q4f)) / T(ray.eta);
            e00 = i0 * ray.n_p4 + k0;
            e10 = i1 * ray.n_p4 + k0;
            e01 = i0 * ray.n_p4 + k1;
            e11 = i1 * ray.n_p4 + k1;
            rconj = q4f < 0.0;
        }
#pragma unroll
        for (int t = 0; t < TB; ++t) {
            if (t < nb) {
                C x[6];  // A, C, B, sv, s4 q~_4, ss at the internal point
                load_point<T>(vec + ((size_t)(b0 + t) * n_int + j) * 12, x);
                const T* d = ext[wib][t];
                const C Ai{d[0], d[1]}, Ci{d[2], d[3]}, Bi{d[4], d[5]};
                C Ad = Ai, Cd = Ci, Bd = Bi;
                if (RAY) {
                    const T u = d[6] * dq4;
                    if (u * u < kRayCut) {  // beta = exp(-u^2) above exp(-39.2), about 1e-17
                        const T beta = exp(-u * u);
                        const int b = list ? list[b0 + t] : b0 + t;
                        const T w00 = (T(1) - ra) * (T(1) - rb), w10 = ra * (T(1) - rb);
                        const T w01 = (T(1) - ra) * rb, w11 = ra * rb;
                        C* dst[3] = {&Ad, &Cd, &Bd};
                        const C own[3] = {Ai, Ci, Bi};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const double* Fc = F_ext + ((size_t)b * 3 + c) * 2 * n_ext;
                            T xr = T(Fc[2 * e00]) * w00 + T(Fc[2 * e10]) * w10;
                            T xi = T(Fc[2 * e00 + 1]) * w00 + T(Fc[2 * e10 + 1]) * w10;
                            xr = xr + T(Fc[2 * e01]) * w01;
                            xi = xi + T(Fc[2 * e01 + 1]) * w01;
                            xr = xr + T(Fc[2 * e11]) * w11;
                            xi = xi + T(Fc[2 * e11 + 1]) * w11;
                            if (rconj) xi = -xi;
                            *dst[c] = C{own[c].re + beta * (xr - own[c].re),
                                        own[c].im + beta * (xi - own[c].im)};
                        }
                    }
                }
                qmu::mu_pair_add_dq<T>(pr, s, d[6], bc != 0, Ai, Ci, Bi, Ad, Cd, Bd, x[0], x[1],
                                       x[2], x[3], x[4], x[5], SA[t], SC[t], SB[t]);
            }
        }
    }
    // warp all-reduce of the 6 TB sums; lane t writes chemical potential b0 + t
#pragma unroll
    for (int t = 0; t < TB; ++t) {
        T y[6] = {SA[t].re, SA[t].im, SC[t].re, SC[t].im, SB[t].re, SB[t].im};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y[c] += __shfl_xor_sync(0xffffffffu, y[c], o);
        }
        if (lane == t && t < nb) {
            const int b = list ? list[b0 + t] : b0 + t;
            const double sa_re = kappa * (double)y[0], sa_im = kappa * (double)y[1];
            const double sc_re = kappa * (double)y[2], sc_im = kappa * (double)y[3];
            const double sb_re = kappa * (double)y[4], sb_im = kappa * (double)y[5];
            // C = 1 + S_C / p~_4
            const double pr_ = row.p4, pi_ = mu[b], dd = 1.0 / (pr_ * pr_ + pi_ * pi_);
            double* Fo = F_out + (size_t)b * 6 * n_ext;
            Fo[2 * e] = 1.0 + sa_re;
            Fo[2 * e + 1] = sa_im;
            Fo[2 * n_ext + 2 * e] = 1.0 + (sc_re * pr_ + sc_im * pi_) * dd;
            Fo[2 * n_ext + 2 * e + 1] = (sc_im * pr_ - sc_re * pi_) * dd;
            Fo[4 * n_ext + 2 * e] = m_cur + sb_re;
            Fo[4 * n_ext + 2 * e + 1] = sb_im;
        }
    }
}

bool finite_all(const double* x, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

bool increasing(const double* x, int n) {
    for (int i = 1; i < n; ++i)
        if (!(x[i] > x[i - 1])) return false;
    return true;
}

}  // namespace

struct qdse_mu_grid {
    int n_ext = 0, n_r = 0, n_4 = 0, n_int = 0, nz = 0, precision = QDSE_FP64;
    double omega = 0;
    long long n_pairs = 0;
    size_t elem = 8;
    MuRow* rows = nullptr;
    double *qr = nullptr, *q4 = nullptr, *wq = nullptr, *z = nullptr, *wz = nullptr;
    void* table = nullptr;
    void* vec = nullptr;
    double* mu = nullptr;
    int mu_cap = 0;
    // external product grid and interpolation onto the internal points (create_product only)
    int n_pr = 0, n_p4 = 0;
    MuInterp* interp = nullptr;
    double *pax = nullptr, *p4ax = nullptr;  // the product grid's axes (reading M8's ray points)
    double ray_eta = 0.0;                     // reading M8 on (> 0, GeV^2) or off (0)
    double fingerprint = 0;  // of every node and weight: grids with equal points match
    // solve workspace: the new iterate, per-mu change, non-finite and done flags
    double* G = nullptr;
    double* change = nullptr;
    int *bad = nullptr, *done = nullptr;
    int solve_cap = 0;     // capacity (chemical potentials) of G, change, bad, done
    int* list = nullptr;  // chemical potentials this grid sweeps in the current step
    int list_cap = 0;
    // profiling: event triples (before prep, between, after sweep) of unread calls
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    int n_rec = 0;
};

extern "C" {

const char* qdse_mu_last_error(void) { return g_mu_err.c_str(); }

void qdse_mu_grid_destroy(qdse_mu_grid* g) {
    if (!g) return;
    for (void* p : {(void*)g->rows, (void*)g->qr, (void*)g->q4, (void*)g->wq, (void*)g->z,
                    (void*)g->wz, g->table, g->vec, (void*)g->mu, (void*)g->interp,
                    (void*)g->pax, (void*)g->p4ax, (void*)g->G,
                    (void*)g->change, (void*)g->bad, (void*)g->done, (void*)g->list})
        if (p) cudaFree(p);
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    delete g;
}

int qdse_mu_grid_create(int n_ext, const double* p_abs, const double* p4, int n_r,
                        const double* q_abs, int n_4, const double* q4, const double* w_q, int n_z,
                        const double* z, const double* w_z, double omega, int precision,
                        void* stream, qdse_mu_grid** out) {
    if (!out) return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: out is NULL");
    *out = nullptr;
    if (n_ext < 1 || n_r < 1 || n_4 < 1 || n_z < 1)
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: n_ext, n_r, n_4, n_z must be >= 1");
    if (n_z > kMaxZ) return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: n_z above %d", kMaxZ);
    if ((long long)n_r * n_4 > (1LL << 28))
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: n_r * n_4 above 2^28");
    if (!p_abs || !p4 || !q_abs || !q4 || !w_q || !z || !w_z)
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: NULL array");
    if (!(omega > 0) || !std::isfinite(omega))
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: omega must be finite and > 0");
    if (precision != QDSE_FP64 && precision != QDSE_FP32)
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: precision must be QDSE_FP64 or QDSE_FP32");
    const int n_int = n_r * n_4;
    if (!finite_all(p_abs, n_ext) || !finite_all(p4, n_ext) || !finite_all(q_abs, n_r) ||
        !finite_all(q4, n_4) || !finite_all(w_q, n_int) || !finite_all(z, n_z) ||
        !finite_all(w_z, n_z))
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: non-finite node or weight");
    for (int e = 0; e < n_ext; ++e)
        if (!(p_abs[e] > 0)) return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: p_abs must be > 0");
    if (!(q_abs[0] > 0) || !increasing(q_abs, n_r) || !increasing(q4, n_4))
        return mu_fail(QDSE_ERR_ARG,
                       "qdse_mu_grid_create: q_abs (> 0) and q4 must be strictly increasing");
    for (int k = 0; k < n_z; ++k)
        if (!(z[k] > -1.0 && z[k] < 1.0))
            return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create: z nodes must lie in (-1, 1)");

    // windows: |P - Q| <= L and |p_4 - q_4| <= L, L^2 = 70 omega^2 (outside, every angle's
    // Gaussian factor is below exp(-70))
    const double L = std::sqrt(qmu::kSkipExponent) * omega;
    std::vector<MuRow> rows(n_ext);
    long long off = 0;
    for (int e = 0; e < n_ext; ++e) {
        MuRow& w = rows[e];
        const int r_lo = (int)(std::lower_bound(q_abs, q_abs + n_r, p_abs[e] - L) - q_abs);
        const int r_hi = (int)(std::upper_bound(q_abs, q_abs + n_r, p_abs[e] + L) - q_abs);
        const int f_lo = (int)(std::lower_bound(q4, q4 + n_4, p4[e] - L) - q4);
        const int f_hi = (int)(std::upper_bound(q4, q4 + n_4, p4[e] + L) - q4);
        const int nr = std::max(0, r_hi - r_lo), nf = std::max(0, f_hi - f_lo);
        w.off = off;
        w.len = nr * nf;
        w.r_lo = std::min(r_lo, n_r - 1);
        w.f_lo = std::min(f_lo, n_4 - 1);
        w.nf = std::max(nf, 1);
        w.P = p_abs[e];
        w.p4 = p4[e];
        off += w.len;
    }

    qdse_mu_grid* g = new qdse_mu_grid;
    g->n_ext = n_ext;
    g->n_r = n_r;
    g->n_4 = n_4;
    g->n_int = n_int;
    g->nz = n_z;
    g->precision = precision;
    g->omega = omega;
    g->n_pairs = off;
    g->elem = precision == QDSE_FP32 ? sizeof(float) : sizeof(double);
    {
        double fp = omega;
        auto mix = [&](const double* x, int n) {
            for (int i = 0; i < n; ++i) fp += x[i] * (1.0 + 1e-3 * (i % 97));
        };
        mix(p_abs, n_ext);
        mix(p4, n_ext);
        mix(q_abs, n_r);
        mix(q4, n_4);
        mix(w_q, n_int);
        mix(z, n_z);
        mix(w_z, n_z);
        g->fingerprint = fp;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = QDSE_OK;
    auto alloc = [&](void** p, size_t bytes, const char* what) {
        if (rc == QDSE_OK) rc = mu_cuda(cudaMalloc(p, std::max<size_t>(bytes, 16)), what);
    };
    alloc((void**)&g->rows, sizeof(MuRow) * n_ext, "cudaMalloc(rows)");
    alloc((void**)&g->qr, sizeof(double) * n_r, "cudaMalloc(q_abs)");
    alloc((void**)&g->q4, sizeof(double) * n_4, "cudaMalloc(q4)");
    alloc((void**)&g->wq, sizeof(double) * n_int, "cudaMalloc(w_q)");
    alloc((void**)&g->z, sizeof(double) * n_z, "cudaMalloc(z)");
    alloc((void**)&g->wz, sizeof(double) * n_z, "cudaMalloc(w_z)");
    alloc(&g->table, g->elem * qmu::kPlanes * (size_t)off, "cudaMalloc(moment table)");
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (rc == QDSE_OK)
            rc = mu_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st),
                         "cudaMemcpyAsync(grid)");
    };
    put(g->rows, rows.data(), sizeof(MuRow) * n_ext);
    put(g->qr, q_abs, sizeof(double) * n_r);
    put(g->q4, q4, sizeof(double) * n_4);
    put(g->wq, w_q, sizeof(double) * n_int);
    put(g->z, z, sizeof(double) * n_z);
    put(g->wz, w_z, sizeof(double) * n_z);
    if (rc == QDSE_OK && off > 0) {
        // constant part of measure x interaction: 2 pi/(2 pi)^4 x 8 pi^2/omega^4 = 1/(pi omega^4)
        const double scale = 1.0 / (kPi * omega * omega * omega * omega);
        const size_t smem = 2 * sizeof(double) * n_z;
        if (precision == QDSE_FP32)
            k_mu_moments<float><<<n_ext, kMomentThreads, smem, st>>>(
                g->rows, g->qr, g->q4, g->wq, n_4, n_z, g->z, g->wz, omega, scale,
                (float*)g->table);
        else
            k_mu_moments<double><<<n_ext, kMomentThreads, smem, st>>>(
                g->rows, g->qr, g->q4, g->wq, n_4, n_z, g->z, g->wz, omega, scale,
                (double*)g->table);
        rc = mu_cuda(cudaGetLastError(), "k_mu_moments launch");
    }
    // the host rows vector is freed on return: wait for its copy
    if (rc == QDSE_OK) rc = mu_cuda(cudaStreamSynchronize(st), "qdse_mu_grid_create");
    if (rc != QDSE_OK) {
        qdse_mu_grid_destroy(g);
        return rc;
    }
    *out = g;
    return QDSE_OK;
}

int qdse_mu_grid_info(const qdse_mu_grid* g, long long* n_pairs, long long* table_bytes) {
    if (!g) return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_info: grid is NULL");
    if (n_pairs) *n_pairs = g->n_pairs;
    if (table_bytes) *table_bytes = (long long)(g->elem * qmu::kPlanes * g->n_pairs);
    return QDSE_OK;
}

}  // extern "C"

namespace {

int check_physics(const char* who, int n_mu, const double* mu, double D, double m, double cf,
                  int vertex) {
    if (vertex != QDSE_VERTEX_BC && vertex != QDSE_VERTEX_RL)
        return mu_fail(QDSE_ERR_ARG, "%s: vertex must be BC or RL", who);
    if (!std::isfinite(D) || !std::isfinite(m) || !std::isfinite(cf))
        return mu_fail(QDSE_ERR_ARG, "%s: D, m, cf must be finite", who);
    if (!finite_all(mu, n_mu)) return mu_fail(QDSE_ERR_ARG, "%s: non-finite mu", who);
    for (int b = 0; b < n_mu; ++b)
        if (mu[b] < 0) return mu_fail(QDSE_ERR_ARG, "%s: mu must be >= 0", who);
    return QDSE_OK;
}

// Grows the per-mu workspace of g to n_mu and uploads the chemical potentials.
int mu_workspace(qdse_mu_grid* g, int n_mu, const double* mu, cudaStream_t st) {
    if (n_mu > g->mu_cap) {
        // the stream's earlier work may still read the old buffers
        int rc = mu_cuda(cudaStreamSynchronize(st), "mu workspace (grow)");
        if (rc != QDSE_OK) return rc;
        if (g->vec) cudaFree(g->vec);
        if (g->mu) cudaFree(g->mu);
        g->vec = nullptr;
        g->mu = nullptr;
        g->mu_cap = 0;
        rc = mu_cuda(cudaMalloc(&g->vec, g->elem * 12 * (size_t)g->n_int * n_mu),
                     "cudaMalloc(mu workspace)");
        if (rc == QDSE_OK) rc = mu_cuda(cudaMalloc((void**)&g->mu, sizeof(double) * n_mu),
                                        "cudaMalloc(mu values)");
        if (rc != QDSE_OK) return rc;
        g->mu_cap = n_mu;
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    return mu_cuda(cudaMemcpyAsync(g->mu, mu, sizeof(double) * n_mu, cudaMemcpyHostToDevice, st),
                   "cudaMemcpyAsync(mu)");
}

// prep (from F_int, or interpolated from F_ext when F_int is NULL) + sweep, on stream st.
// list: NULL (chemical potentials 0 .. n_mu-1) or device int[n_mu] (interpolated prep only).
int mu_launch(qdse_mu_grid* g, int n_mu, const int* list, double D, double m, double cf,
              int vertex, const double* F_ext, const double* F_int, double* F_out,
              cudaStream_t st) {
    const size_t total = (size_t)n_mu * g->n_int;
    const int prep_blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    const double kappa = cf * D;
    const int bc = vertex == QDSE_VERTEX_BC;
    RayArgs ray{g->pax, g->p4ax, g->n_pr, g->n_p4, 0.0};
    if (g->ray_eta > 0.0 && g->pax && bc) ray.eta = g->ray_eta;
    cudaEvent_t* evt = nullptr;
    if (g->profiling) {
        if ((size_t)(3 * g->n_rec + 3) > g->ev.size()) {
            for (int k = 0; k < 3; ++k) {
                cudaEvent_t e;
                const int rc = mu_cuda(cudaEventCreate(&e), "cudaEventCreate");
                if (rc != QDSE_OK) return rc;
                g->ev.push_back(e);
            }
        }
        evt = &g->ev[3 * g->n_rec];
        g->n_rec++;
    }
    auto mark = [&](int k) {
        if (evt) cudaEventRecord(evt[k], st);
    };
    mark(0);
    if (g->precision == QDSE_FP32) {
        if (F_int)
            k_mu_prep<float><<<prep_blocks, 256, 0, st>>>(n_mu, g->mu, g->n_int, g->n_4, g->qr,
                                                          g->q4, F_int, (float*)g->vec);
        else
            k_mu_prep_interp<float><<<prep_blocks, 256, 0, st>>>(
                n_mu, list, g->mu, g->n_int, g->n_4, g->qr, g->q4, g->interp, F_ext, g->n_ext,
                (float*)g->vec);
        mark(1);
        const int n_tiles = (n_mu + kTileF32 - 1) / kTileF32;
        const long long warps = (long long)g->n_ext * n_tiles;
        const unsigned blocks = (unsigned)((warps + 3) / 4);
        if (ray.eta > 0.0)
            k_mu_sweep<float, kTileF32, 4, true><<<blocks, kSweepThreads, 0, st>>>(
                g->rows, g->qr, g->q4, (const float*)g->table, (const float*)g->vec, g->n_int,
                g->n_4, n_mu, list, n_tiles, g->mu, F_ext, g->n_ext, kappa, m, bc, F_out, ray);
        else
            k_mu_sweep<float, kTileF32, 4, false><<<blocks, kSweepThreads, 0, st>>>(
                g->rows, g->qr, g->q4, (const float*)g->table, (const float*)g->vec, g->n_int,
                g->n_4, n_mu, list, n_tiles, g->mu, F_ext, g->n_ext, kappa, m, bc, F_out, ray);
    } else {
        if (F_int)
            k_mu_prep<double><<<prep_blocks, 256, 0, st>>>(n_mu, g->mu, g->n_int, g->n_4, g->qr,
                                                           g->q4, F_int, (double*)g->vec);
        else
            k_mu_prep_interp<double><<<prep_blocks, 256, 0, st>>>(
                n_mu, list, g->mu, g->n_int, g->n_4, g->qr, g->q4, g->interp, F_ext, g->n_ext,
                (double*)g->vec);
        mark(1);
        const int n_tiles = (n_mu + kTileF64 - 1) / kTileF64;
        const long long warps = (long long)g->n_ext * n_tiles;
        const unsigned blocks = (unsigned)((warps + 3) / 4);
        if (ray.eta > 0.0)
            k_mu_sweep<double, kTileF64, 2, true><<<blocks, kSweepThreads, 0, st>>>(
                g->rows, g->qr, g->q4, (const double*)g->table, (const double*)g->vec, g->n_int,
                g->n_4, n_mu, list, n_tiles, g->mu, F_ext, g->n_ext, kappa, m, bc, F_out, ray);
        else
            k_mu_sweep<double, kTileF64, 2, false><<<blocks, kSweepThreads, 0, st>>>(
                g->rows, g->qr, g->q4, (const double*)g->table, (const double*)g->vec, g->n_int,
                g->n_4, n_mu, list, n_tiles, g->mu, F_ext, g->n_ext, kappa, m, bc, F_out, ray);
    }
    mark(2);
    return mu_cuda(cudaGetLastError(), "finite-mu sweep launch");
}

// Reading M6 on the host: (lower index, weight of the upper node) of x on an ascending axis;
// held at the first/last node outside it.
void bracket(const double* axis, int n, double x, int* i, double* w) {
    const int k = (int)(std::upper_bound(axis, axis + n, x) - axis) - 1;
    if (k < 0) {
        *i = 0;
        *w = 0.0;
    } else if (k >= n - 1) {
        *i = n - 1;
        *w = 0.0;
    } else {
        *i = k;
        *w = (x - axis[k]) / (axis[k + 1] - axis[k]);
    }
}

}  // namespace

extern "C" {

int qdse_mu_sweep(qdse_mu_grid* g, int n_mu, const double* mu, double D, double m, double cf,
                  int vertex, const double* F_ext, const double* F_int, double* F_out,
                  void* stream) {
    if (!g) return mu_fail(QDSE_ERR_ARG, "qdse_mu_sweep: grid is NULL");
    if (n_mu < 0) return mu_fail(QDSE_ERR_ARG, "qdse_mu_sweep: n_mu < 0");
    if (n_mu == 0) return QDSE_OK;
    if ((long long)g->n_ext * ((n_mu + kTileF64 - 1) / kTileF64) > (1LL << 32))
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_sweep: n_ext * n_mu too large for one launch");
    if (!mu || !F_ext || !F_int || !F_out) return mu_fail(QDSE_ERR_ARG, "qdse_mu_sweep: NULL array");
    int rc = check_physics("qdse_mu_sweep", n_mu, mu, D, m, cf, vertex);
    if (rc != QDSE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = mu_workspace(g, n_mu, mu, st);
    if (rc != QDSE_OK) return rc;
    return mu_launch(g, n_mu, nullptr, D, m, cf, vertex, F_ext, F_int, F_out, st);
}

int qdse_mu_grid_create_product(int n_pr, const double* p_axis, int n_p4, const double* p4_axis,
                                int n_r, const double* q_abs, int n_4, const double* q4,
                                const double* w_q, int n_z, const double* z, const double* w_z,
                                double omega, int precision, void* stream, qdse_mu_grid** out) {
    if (!out) return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create_product: out is NULL");
    *out = nullptr;
    if (n_pr < 1 || n_p4 < 1 || !p_axis || !p4_axis)
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create_product: empty or NULL axis");
    if ((long long)n_pr * n_p4 > (1LL << 28))
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_grid_create_product: n_pr * n_p4 above 2^28");
    if (!finite_all(p_axis, n_pr) || !finite_all(p4_axis, n_p4) || !(p_axis[0] > 0) ||
        !(p4_axis[0] > 0) || !increasing(p_axis, n_pr) || !increasing(p4_axis, n_p4))
        return mu_fail(QDSE_ERR_ARG,
                       "qdse_mu_grid_create_product: axes must be finite, > 0 and strictly "
                       "increasing");
    const int n_ext = n_pr * n_p4;
    std::vector<double> pa(n_ext), p4a(n_ext);
    for (int i = 0; i < n_pr; ++i)
        for (int k = 0; k < n_p4; ++k) {
            pa[(size_t)i * n_p4 + k] = p_axis[i];
            p4a[(size_t)i * n_p4 + k] = p4_axis[k];
        }
    qdse_mu_grid* g = nullptr;
    int rc = qdse_mu_grid_create(n_ext, pa.data(), p4a.data(), n_r, q_abs, n_4, q4, w_q, n_z, z,
                                 w_z, omega, precision, stream, &g);
    if (rc != QDSE_OK) return rc;
    std::vector<MuInterp> ip((size_t)n_r * n_4);
    for (int r = 0; r < n_r; ++r)
        for (int f = 0; f < n_4; ++f) {
            int i, k;
            double a, b;
            bracket(p_axis, n_pr, q_abs[r], &i, &a);
            bracket(p4_axis, n_p4, std::fabs(q4[f]), &k, &b);
            const int i1 = std::min(i + 1, n_pr - 1), k1 = std::min(k + 1, n_p4 - 1);
            MuInterp& e = ip[(size_t)r * n_4 + f];
            e.e00 = i * n_p4 + k;
            e.e10 = i1 * n_p4 + k;
            e.e01 = i * n_p4 + k1;
            e.e11 = i1 * n_p4 + k1;
            e.a = a;
            e.b = b;
            e.conj = q4[f] < 0;
            e.pad = 0;
        }
    cudaStream_t st = (cudaStream_t)stream;
    rc = mu_cuda(cudaMalloc((void**)&g->interp, sizeof(MuInterp) * ip.size()),
                 "cudaMalloc(interpolation)");
    if (rc == QDSE_OK)
        rc = mu_cuda(cudaMemcpyAsync(g->interp, ip.data(), sizeof(MuInterp) * ip.size(),
                                     cudaMemcpyHostToDevice, st),
                     "cudaMemcpyAsync(interpolation)");
    if (rc == QDSE_OK) rc = mu_cuda(cudaMalloc((void**)&g->pax, sizeof(double) * n_pr), "cudaMalloc(axis)");
    if (rc == QDSE_OK) rc = mu_cuda(cudaMalloc((void**)&g->p4ax, sizeof(double) * n_p4), "cudaMalloc(axis)");
    if (rc == QDSE_OK)
        rc = mu_cuda(cudaMemcpyAsync(g->pax, p_axis, sizeof(double) * n_pr, cudaMemcpyHostToDevice,
                                     st), "cudaMemcpyAsync(axis)");
    if (rc == QDSE_OK)
        rc = mu_cuda(cudaMemcpyAsync(g->p4ax, p4_axis, sizeof(double) * n_p4,
                                     cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(axis)");
    if (rc == QDSE_OK) rc = mu_cuda(cudaStreamSynchronize(st), "qdse_mu_grid_create_product");
    if (rc != QDSE_OK) {
        qdse_mu_grid_destroy(g);
        return rc;
    }
    g->n_pr = n_pr;
    g->n_p4 = n_p4;
    *out = g;
    return QDSE_OK;
}

int qdse_mu_solve(qdse_mu_grid* g, qdse_mu_grid* refine, int n_mu, const double* mu, double D,
                  double m, double cf, int vertex, double alpha, double tol, double switch_tol,
                  int max_iter, double* F, int* iters, int* status, void* stream) {
    const char* who = "qdse_mu_solve";
    if (!g) return mu_fail(QDSE_ERR_ARG, "%s: grid is NULL", who);
    if (!g->interp)
        return mu_fail(QDSE_ERR_ARG, "%s: the grid was not made by qdse_mu_grid_create_product",
                       who);
    if (refine && (!refine->interp || refine->n_ext != g->n_ext || refine->n_int != g->n_int ||
                   refine->fingerprint != g->fingerprint))
        return mu_fail(QDSE_ERR_ARG, "%s: refine must be a product grid on the same points", who);
    if (n_mu < 0) return mu_fail(QDSE_ERR_ARG, "%s: n_mu < 0", who);
    if (n_mu == 0) return QDSE_OK;
    if ((long long)g->n_ext * ((n_mu + kTileF64 - 1) / kTileF64) > (1LL << 32))
        return mu_fail(QDSE_ERR_ARG, "%s: n_ext * n_mu too large for one launch", who);
    if (!mu || !F) return mu_fail(QDSE_ERR_ARG, "%s: NULL array", who);
    if (!(alpha > 0 && alpha <= 1)) return mu_fail(QDSE_ERR_ARG, "%s: alpha must be in (0, 1]", who);
    if (!(tol >= 0) || !std::isfinite(tol) || !(switch_tol >= 0) || !std::isfinite(switch_tol))
        return mu_fail(QDSE_ERR_ARG, "%s: tol and switch_tol must be finite and >= 0", who);
    if (max_iter < 1) return mu_fail(QDSE_ERR_ARG, "%s: max_iter must be >= 1", who);
    int rc = check_physics(who, n_mu, mu, D, m, cf, vertex);
    if (rc != QDSE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = mu_workspace(g, n_mu, mu, st);
    if (rc == QDSE_OK && refine) rc = mu_workspace(refine, n_mu, mu, st);
    if (rc != QDSE_OK) return rc;
    // the stream's earlier work may still read the buffers about to be replaced
    auto grow_list = [&](qdse_mu_grid* x) -> int {
        if (n_mu <= x->list_cap) return QDSE_OK;
        int r = mu_cuda(cudaStreamSynchronize(st), "qdse_mu_solve (grow)");
        if (r != QDSE_OK) return r;
        if (x->list) cudaFree(x->list);
        x->list = nullptr;
        x->list_cap = 0;
        r = mu_cuda(cudaMalloc((void**)&x->list, sizeof(int) * n_mu), "cudaMalloc(list)");
        if (r == QDSE_OK) x->list_cap = n_mu;
        return r;
    };
    rc = grow_list(g);
    if (rc == QDSE_OK && refine) rc = grow_list(refine);
    if (rc != QDSE_OK) return rc;
    if (n_mu > g->solve_cap) {
        rc = mu_cuda(cudaStreamSynchronize(st), "qdse_mu_solve (grow)");
        if (rc != QDSE_OK) return rc;
        for (void* p : {(void*)g->G, (void*)g->change, (void*)g->bad, (void*)g->done})
            if (p) cudaFree(p);
        g->G = nullptr;
        g->change = nullptr;
        g->bad = g->done = nullptr;
        g->solve_cap = 0;
        rc = mu_cuda(cudaMalloc((void**)&g->G, sizeof(double) * 6 * (size_t)g->n_ext * n_mu),
                     "cudaMalloc(solve workspace)");
        if (rc == QDSE_OK)
            rc = mu_cuda(cudaMalloc((void**)&g->change, sizeof(double) * n_mu), "cudaMalloc");
        if (rc == QDSE_OK) rc = mu_cuda(cudaMalloc((void**)&g->bad, sizeof(int) * n_mu), "cudaMalloc");
        if (rc == QDSE_OK) rc = mu_cuda(cudaMalloc((void**)&g->done, sizeof(int) * n_mu), "cudaMalloc");
        if (rc != QDSE_OK) return rc;
        g->solve_cap = n_mu;
    }
    std::vector<int> done(n_mu, 0), bad(n_mu, 0), it_at(n_mu, 0), phase(n_mu, 0);
    std::vector<int> bad_now(n_mu, 0), list0, list1;
    std::vector<double> change(n_mu, 0.0);
    // per chemical potential: phase 0 sweeps on g (to switch_tol when refining, else to tol),
    // phase 1 sweeps on refine (to tol); converged or non-finite ones are no longer swept
    int it = 0;
    while (it < max_iter) {
        ++it;
        list0.clear();
        list1.clear();
        for (int b = 0; b < n_mu; ++b)
            if (!done[b]) (phase[b] == 0 ? list0 : list1).push_back(b);
        if (list0.empty() && list1.empty()) break;
        rc = mu_cuda(cudaMemcpyAsync(g->done, done.data(), sizeof(int) * n_mu,
                                     cudaMemcpyHostToDevice, st),
                     "cudaMemcpyAsync(done)");
        if (rc == QDSE_OK && !list0.empty()) {
            rc = mu_cuda(cudaMemcpyAsync(g->list, list0.data(), sizeof(int) * list0.size(),
                                         cudaMemcpyHostToDevice, st),
                         "cudaMemcpyAsync(list)");
            if (rc == QDSE_OK)
                rc = mu_launch(g, (int)list0.size(), g->list, D, m, cf, vertex, F, nullptr, g->G,
                               st);
        }
        if (rc == QDSE_OK && !list1.empty()) {
            rc = mu_cuda(cudaMemcpyAsync(refine->list, list1.data(), sizeof(int) * list1.size(),
                                         cudaMemcpyHostToDevice, st),
                         "cudaMemcpyAsync(list)");
            if (rc == QDSE_OK)
                rc = mu_launch(refine, (int)list1.size(), refine->list, D, m, cf, vertex, F,
                               nullptr, g->G, st);
        }
        if (rc != QDSE_OK) return rc;
        k_mu_relax<<<n_mu, kRelaxThreads, 0, st>>>(g->n_ext, alpha, F, g->G, g->done, g->change,
                                                   g->bad);
        rc = mu_cuda(cudaGetLastError(), "k_mu_relax launch");
        if (rc == QDSE_OK)
            rc = mu_cuda(cudaMemcpyAsync(change.data(), g->change, sizeof(double) * n_mu,
                                         cudaMemcpyDeviceToHost, st),
                         "cudaMemcpyAsync(change)");
        if (rc == QDSE_OK)
            rc = mu_cuda(cudaMemcpyAsync(bad_now.data(), g->bad, sizeof(int) * n_mu,
                                         cudaMemcpyDeviceToHost, st),
                         "cudaMemcpyAsync(bad)");
        if (rc == QDSE_OK) rc = mu_cuda(cudaStreamSynchronize(st), who);
        if (rc != QDSE_OK) return rc;
        for (int b = 0; b < n_mu; ++b) {
            if (done[b]) continue;
            if (bad_now[b]) {
                bad[b] = 1;
                done[b] = 1;  // frozen from here on
            } else if (refine && phase[b] == 0) {
                if (change[b] < std::max(tol, switch_tol)) phase[b] = 1;
            } else if (change[b] < tol) {
                done[b] = 1;
                it_at[b] = it;
            }
        }
    }
    for (int b = 0; b < n_mu; ++b) {
        if (iters) iters[b] = done[b] && !bad[b] ? it_at[b] : it;
        if (status)
            status[b] = bad[b] ? QDSE_ERR_NONFINITE : done[b] ? QDSE_OK : QDSE_ERR_NOT_CONVERGED;
    }
    return QDSE_OK;
}

int qdse_mu_solve_continued(qdse_mu_grid* g, qdse_mu_grid* refine, int n_mu, const double* mu,
                            double D, double m, double cf, int vertex, double alpha, double tol,
                            double switch_tol, int max_iter, int max_rounds, double* F,
                            int* iters, int* status, int* rounds, void* stream) {
    const char* who = "qdse_mu_solve_continued";
    if (max_rounds < 1) return mu_fail(QDSE_ERR_ARG, "%s: max_rounds must be >= 1", who);
    if (n_mu < 0) return mu_fail(QDSE_ERR_ARG, "%s: n_mu < 0", who);
    if (n_mu == 0) return QDSE_OK;
    if (!mu || !F) return mu_fail(QDSE_ERR_ARG, "%s: NULL array", who);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> it_all(n_mu, 0), st_all(n_mu, QDSE_ERR_NOT_CONVERGED), rnd(n_mu, 0);
    std::vector<int> from(n_mu, -1);  // the converged neighbour the last attempt started from
    // round 0: every chemical potential from the caller's start
    int rc = qdse_mu_solve(g, refine, n_mu, mu, D, m, cf, vertex, alpha, tol, switch_tol, max_iter,
                           F, it_all.data(), st_all.data(), stream);
    if (rc != QDSE_OK) return rc;
    const size_t fbytes = sizeof(double) * 6 * (size_t)g->n_ext;  // one mu's A, C, B
    double* sub = nullptr;
    for (int r = 1; r < max_rounds; ++r) {
        // each unconverged mu restarts from its nearest converged neighbour in mu (the lower one on
        // a tie), unless that is the neighbour its last attempt already started from
        std::vector<int> pick, nb;
        for (int b = 0; b < n_mu; ++b) {
            if (st_all[b] == QDSE_OK) continue;
            int best = -1;
            for (int c = 0; c < n_mu; ++c) {
                if (st_all[c] != QDSE_OK) continue;
                const double d = std::fabs(mu[c] - mu[b]);
                const double e = best < 0 ? 0.0 : std::fabs(mu[best] - mu[b]);
                if (best < 0 || d < e || (d == e && mu[c] < mu[best])) best = c;
            }
            if (best >= 0 && best != from[b]) {
                pick.push_back(b);
                nb.push_back(best);
            }
        }
        if (pick.empty()) break;
        const int n_sub = (int)pick.size();
        if (!sub) {
            rc = mu_cuda(cudaMalloc((void**)&sub, fbytes * n_mu), "cudaMalloc(continuation)");
            if (rc != QDSE_OK) return rc;
        }
        std::vector<double> mu_sub(n_sub);
        for (int k = 0; k < n_sub && rc == QDSE_OK; ++k) {
            mu_sub[k] = mu[pick[k]];
            rc = mu_cuda(cudaMemcpyAsync(sub + (size_t)k * 6 * g->n_ext,
                                         F + (size_t)nb[k] * 6 * g->n_ext, fbytes,
                                         cudaMemcpyDeviceToDevice, st),
                         "cudaMemcpyAsync(continuation start)");
        }
        std::vector<int> it_sub(n_sub), st_sub(n_sub);
        if (rc == QDSE_OK)
            rc = qdse_mu_solve(g, refine, n_sub, mu_sub.data(), D, m, cf, vertex, alpha, tol,
                               switch_tol, max_iter, sub, it_sub.data(), st_sub.data(), stream);
        for (int k = 0; k < n_sub && rc == QDSE_OK; ++k) {
            const int b = pick[k];
            from[b] = nb[k];
            it_all[b] += it_sub[k];
            rnd[b] = r;
            // a converged restart replaces the iterate; a failed one leaves the last attempt's
            if (st_sub[k] == QDSE_OK || st_all[b] == QDSE_ERR_NONFINITE) {
                st_all[b] = st_sub[k];
                rc = mu_cuda(cudaMemcpyAsync(F + (size_t)b * 6 * g->n_ext,
                                             sub + (size_t)k * 6 * g->n_ext, fbytes,
                                             cudaMemcpyDeviceToDevice, st),
                             "cudaMemcpyAsync(continuation result)");
            }
        }
        if (rc != QDSE_OK) break;
    }
    if (sub) {
        const int r2 = mu_cuda(cudaStreamSynchronize(st), who);
        cudaFree(sub);
        if (rc == QDSE_OK) rc = r2;
    }
    if (rc != QDSE_OK) return rc;
    for (int b = 0; b < n_mu; ++b) {
        if (iters) iters[b] = it_all[b];
        if (status) status[b] = st_all[b];
        if (rounds) rounds[b] = rnd[b];
    }
    return QDSE_OK;
}

int qdse_mu_set_ray_quotient(qdse_mu_grid* g, double eta) {
    if (!g) return mu_fail(QDSE_ERR_ARG, "qdse_mu_set_ray_quotient: grid is NULL");
    if (!g->pax)
        return mu_fail(QDSE_ERR_ARG,
                       "qdse_mu_set_ray_quotient: the grid was not made by "
                       "qdse_mu_grid_create_product");
    if (!(eta >= 0) || !std::isfinite(eta))
        return mu_fail(QDSE_ERR_ARG, "qdse_mu_set_ray_quotient: eta must be finite and >= 0");
    g->ray_eta = eta;
    return QDSE_OK;
}

int qdse_mu_set_profiling(qdse_mu_grid* g, int on) {
    if (!g) return mu_fail(QDSE_ERR_ARG, "qdse_mu_set_profiling: grid is NULL");
    g->profiling = on != 0;
    return QDSE_OK;
}

int qdse_mu_profile(qdse_mu_grid* g, double* ms, long long* launches) {
    if (!g) return mu_fail(QDSE_ERR_ARG, "qdse_mu_profile: grid is NULL");
    double t[2] = {0, 0};
    if (g->n_rec > 0) {
        int rc = mu_cuda(cudaEventSynchronize(g->ev[3 * g->n_rec - 1]), "cudaEventSynchronize");
        if (rc != QDSE_OK) return rc;
        for (int c = 0; c < g->n_rec; ++c)
            for (int k = 0; k < 2; ++k) {
                float x = 0;
                rc = mu_cuda(cudaEventElapsedTime(&x, g->ev[3 * c + k], g->ev[3 * c + k + 1]),
                             "cudaEventElapsedTime");
                if (rc != QDSE_OK) return rc;
                t[k] += x;
            }
    }
    if (ms) {
        ms[0] = t[0];
        ms[1] = t[1];
    }
    if (launches) launches[0] = launches[1] = g->n_rec;
    g->n_rec = 0;
    return QDSE_OK;
}

}  // extern "C"
