// k_precompute.cu -- angular kernel matrices of the Ball-Chiu gap equation.
//
// After the Dirac traces of Eqs. dsesys/dsesys2 every angular dependence of a sweep sits in three
// kernels that do not depend on A or B:
//   K_n(P_i, Q_j) = 8 pi^2/w^4 sum_k w_k exp(-k^2/w^2) g_n(P_i, Q_j, z_k),   n = 0, T, 3,
//   g_0 = 1,  g_T = 2 P Q (1 - z^2)/k^2,  g_3 = [3 x (P + Q) - 4 x^2 - 2 P Q]/k^2,
//   x = sqrt(P Q) z,  k^2 = (sqrt P - sqrt Q)^2 + 2 sqrt(P Q) (1 - z)  (no cancellation at z -> 1).
// Since P + Q = k^2 + 2x, the numerator of g_3 is 3x k^2 - 2PQ(1 - z^2): g_3 = 3x - g_T exactly, so
// K_3 = 3 sqrt(PQ) sum_k w_k E_k z_k - K_T, free of the cancellation of the numerator near the
// diagonal (P = Q, z -> 1), where it vanishes with k^2.
// The interaction strength D is factored out.  K_T only ever multiplies the difference quotients
// (F(q^2) - F(p^2))/(q^2 - p^2), so the pool stores K_T/(Q_j - P_i) and the sweep multiplies it
// by plain differences; on the collocated diagonal it stores K_T itself.
//
// Every entry is evaluated in FP64 and stored as a double-float pair (hi = fl32(K),
// lo = fl32(K - hi)): the FP32 sweeps read hi, the FP64 residual reads hi + lo (about 48 bits).
// Both pools use the group-tile layout of kpos (qdse_internal.h); the collocated diagonal K_T of
// every row is also kept in a per-point array.
// Optionally the omega-derivatives dK_n/dw (factor -4/w + 2 k^2/w^3 on each term) are stored in a
// second pool for the adjoint's dF/dw.
//
// Work is cut into 32 x 32 tiles of (i, j).  On a collocated grid g_n and k^2 are symmetric in
// P <-> Q, so K_0 and K_3 are symmetric and K_T/(Q - P) is antisymmetric: only tiles with
// J >= I are evaluated, and each writes itself and its transpose (through shared memory, so both
// stores are coalesced).  Staggered grids evaluate every tile.  Tiles whose pairs all have
// (sqrt P - sqrt Q)^2 / w^2 beyond kSkipExponent are written as exact zeros without evaluation.
#include <cmath>
#include <vector>

#include "f2.cuh"
#include "qdse_internal.h"

namespace qdse {

// Pairs with (sqrt P - sqrt Q)^2 / w^2 beyond this are written as exact zeros without
// evaluating the sum.  Every term of such a pair carries exp(-k^2/w^2) <= e^-70 (k^2 >=
// (sqrt P - sqrt Q)^2); the polynomial factors of the integrand and of the weights W_j/(Q A^2 +
// B^2) grow by at most (Q_far / Q_near)^3 <~ 1e6 across the grids and w of interest before the
// Gaussian takes over, so the dropped entries change a row's sum by less than 1e-20 of it, far
// below FP64 resolution.
constexpr double kSkipExponent = 70.0;
// Inside a pair, the angular terms have exponents k^2/w^2 increasing with the node index (1 - z
// increases); once a term's exponent exceeds the first term's by this much, it and every later
// term are below e^-60 of the first, times polynomial ratios (g_n, 1/k^2) of at most about 1e4
// (nodes down to theta = pi/129): the sum stops there.
constexpr double kAngularCut = 60.0;

// Writes one 32 x 32 tile of the three kernel planes into the pool (rows i0.., columns j0..) and,
// for an off-diagonal tile of a collocated grid, its transpose (rows j0.., columns i0..; K_0 and
// K_3 symmetric, K_T/(Q - P) odd).  val(p, idx, h, l) gives the (hi, lo) pair of plane p at tile
// position idx = row * (kTile + 1) + column.  Threads walk the destination in layout order: row
// group rg of the tile, 4-column block cb, stored plane-row slot (plane-row m = slot ^ kswz),
// column inside the block; for full groups consecutive threads write consecutive floats.
template <typename Val>
__device__ __forceinline__ void store_tile(const DevInst& I, const Grid& g, const int4& t,
                                           float* __restrict__ Hi, float* __restrict__ Lo,
                                           bool diag, const Val& val) {
    static_assert(kTile % kRows == 0 && kTile % 4 == 0,
                  "precompute tiles must cover whole row groups and 4-column blocks");
    constexpr int kRun = 3 * kRows * kTile;  // floats of one row group inside the tile
    const int i0 = t.y * kTile, j0 = t.z * kTile;
    const bool coll = (I.mode == QDSE_COLLOCATED);
    const bool mirror = coll && t.z != t.y;
    for (int pass = 0; pass < (mirror ? 2 : 1); ++pass) {
        const int rb0 = pass ? j0 : i0, cb0 = pass ? i0 : j0;
        for (int e = threadIdx.x; e < 3 * kTile * kTile; e += blockDim.x) {
            const int rg = e / kRun, off = e % kRun;
            const int cb = off / (3 * kRows * 4), wq = off % (3 * kRows * 4);
            const int slot = wq >> 2, cc = cb * 4 + (wq & 3);
            const int g0 = rb0 + rg * kRows;
            const int nr = min(kRows, I.n - g0);
            const int j = cb0 + cc;
            if (nr <= 0 || slot >= 3 * nr || j >= I.ld) continue;
            const int m = slot ^ kswz(nr, j >> 2);
            const int rr = rg * kRows + m / 3, p = m % 3, i = rb0 + rr;
            float h = 0.f, l = 0.f;
            if (j < I.n) {
                val(p, pass ? cc * (kTile + 1) + rr : rr * (kTile + 1) + cc, h, l);
                if (pass && p == 1) {
                    h = -h;
                    l = -l;
                }
            }
            const long long idx = kpos(I.k_off, I.n, I.ld, i, p, j);
            Hi[idx] = h;
            Lo[idx] = l;
            if (diag && coll && p == 1 && i == j) g.ktd[I.x_off + i] = h;
        }
    }
}

template <bool WITH_W>
__global__ void __launch_bounds__(256) k_precompute_tiles(const DevInst* __restrict__ inst, Grid g,
                                                          const int4* __restrict__ tiles,
                                                          float* __restrict__ Khi,
                                                          float* __restrict__ Klo,
                                                          float* __restrict__ Kwhi,
                                                          float* __restrict__ Kwlo) {
    extern __shared__ double sm[];
    constexpr int S = kTile * (kTile + 1);  // one padded plane of the result tile
    double* tileK = sm;                     // [set][plane][32][33], set 0 = K, set 1 = dK/dw
    const int4 t = tiles[blockIdx.x];       // instance, tile row, tile column
    const DevInst I = inst[t.x];
    double* sy = tileK + (WITH_W ? 2 : 1) * 3 * S;
    double* sz = sy + I.nt;
    double* ss = sz + I.nt;
    double* sw = ss + I.nt;
    for (int k = threadIdx.x; k < I.nt; k += blockDim.x) {
        sy[k] = g.y[I.t_off + k];
        sz[k] = g.z[I.t_off + k];
        ss[k] = g.s2[I.t_off + k];
        sw[k] = g.wz[I.t_off + k];
    }
    __syncthreads();
    const int i0 = t.y * kTile, j0 = t.z * kTile;
    const double w = I.omega;
    const double iw2 = 1.0 / (w * w);
    const double pref = 8.0 * kPi * kPi / (w * w * w * w);
    const double fw0 = -4.0 / w, fw1 = 2.0 / (w * w * w);
    const bool coll = (I.mode == QDSE_COLLOCATED);
    // is the whole tile beyond the skip threshold?  (sqrt s grows with the index)
    bool skip_tile;
    {
        const int i1 = min(i0 + kTile, I.n) - 1, j1 = min(j0 + kTile, I.n) - 1;
        const double pl = g.rsp[I.x_off + i0], ph = g.rsp[I.x_off + i1];
        const double ql = g.rsq[I.x_off + j0], qh = g.rsq[I.x_off + j1];
        const double gap = fmax(0.0, fmax(ql - ph, pl - qh));
        skip_tile = gap * gap * iw2 >= kSkipExponent;
    }
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int li = e / kTile, lj = e % kTile;
        const int i = i0 + li, j = j0 + lj;
        double K0 = 0.0, KT = 0.0, K3 = 0.0, W0 = 0.0, WT = 0.0, W3 = 0.0;
        if (!skip_tile && i < I.n && j < I.n) {
            const double P = g.sp[I.x_off + i], rP = g.rsp[I.x_off + i];
            const double Q = g.sq[I.x_off + j], rQ = g.rsq[I.x_off + j];
            const double dd = (rP - rQ) * (rP - rQ);
            if (dd * iw2 < kSkipExponent) {
                const double c2 = 2.0 * rP * rQ, x0 = rP * rQ, PQ = P * Q;
                const double ex_last = (dd + c2 * sy[0]) * iw2 + kAngularCut;
                // g_3 = 3x - g_T (see the header): accumulate E against 1 and z and
                // E (1 - z^2)/k^2, then K_T = 2PQ sum(E (1 - z^2)/k^2), K_3 = 3 x0 sum(E z) - K_T
                // (likewise for the w-derivatives, every term times f)
                double Sz = 0.0, St = 0.0, Wz = 0.0, Wt = 0.0;
                for (int k = 0; k < I.nt; ++k) {
                    const double k2 = dd + c2 * sy[k];
                    const double ex = k2 * iw2;
                    if (ex > ex_last) break;
                    const double E = sw[k] * exp(-ex);
                    const double T = E * ss[k] / k2;
                    K0 += E;
                    Sz = fma(E, sz[k], Sz);
                    St += T;
                    if (WITH_W) {
                        const double f = fw0 + fw1 * k2;
                        W0 = fma(E, f, W0);
                        Wz = fma(E * f, sz[k], Wz);
                        Wt = fma(T, f, Wt);
                    }
                }
                KT = 2.0 * PQ * St;
                K3 = 3.0 * x0 * Sz - KT;
                if (WITH_W) {
                    WT = 2.0 * PQ * Wt;
                    W3 = 3.0 * x0 * Wz - WT;
                }
                const double dq = (coll && i == j) ? 1.0 : 1.0 / (Q - P);
                K0 *= pref;
                KT *= pref * dq;
                K3 *= pref;
                if (WITH_W) {
                    W0 *= pref;
                    WT *= pref * dq;
                    W3 *= pref;
                }
            }
        }
        const int o = li * (kTile + 1) + lj;
        tileK[0 * S + o] = K0;
        tileK[1 * S + o] = KT;
        tileK[2 * S + o] = K3;
        if (WITH_W) {
            tileK[3 * S + o] = W0;
            tileK[4 * S + o] = WT;
            tileK[5 * S + o] = W3;
        }
    }
    __syncthreads();
    // store the tile (rows i, columns j) and, for an off-diagonal symmetric tile, its transpose
    for (int set = 0; set < (WITH_W ? 2 : 1); ++set) {
        const double* T = tileK + set * 3 * S;
        store_tile(I, g, t, set ? Kwhi : Khi, set ? Kwlo : Klo, set == 0,
                   [&](int p, int idx, float& h, float& l) {
                       const double v = T[p * S + idx];
                       h = __double2float_rn(v);
                       l = __double2float_rn(v - (double)h);
                   });
    }
}

// ------------------------------------------------------------------------------------------------
// The same kernel matrices on the FP32 pipe.  GB300 issues FP64 at about 1/73 of its FP32 rate, and
// the FP64 kernel above spends nearly all of its time in the FP64 exp and division of every angular
// term.  Here each term is evaluated in double-float arithmetic: a value is the unevaluated sum
// h + l of two floats with |l| <= ulp(h)/2 (48 significant bits, relative precision about 4e-15),
// built from the error-free transformations of a sum (Knuth's TwoSum: a + b = s + e exactly) and of
// a product (with a fused multiply-add, a b = p + e exactly, e = fma(a, b, -p)).  The stored pair
// (hi, lo) is the double-float result itself.
//
// The arithmetic of one pair is qf2::pair_entries (f2.cuh).  Pairs whose first angular term already
// has exp(-k^2/w^2) < e^-87.5 (below the FP32 range) are stored as zeros; the FP64 kernel stores
// values of that order there, which move a sweep's A and B by less than 1e-30 of their values.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_precompute_tiles_f2(const DevInst* __restrict__ inst,
                                                             Grid g,
                                                             const int4* __restrict__ tiles,
                                                             float* __restrict__ Khi,
                                                             float* __restrict__ Klo) {
    extern __shared__ float2 smf[];
    constexpr int S = kTile * (kTile + 1);
    float2* tileK = smf;                      // [plane][32][33] pairs
    const int4 t = tiles[blockIdx.x];
    const DevInst I = inst[t.x];
    float2* ta = tileK + 3 * S;               // exp tables (qf2::exp_neg)
    float2* tb = ta + qf2::kExpA;
    float2* sdy = tb + qf2::kExpB;            // per node: y_k - y_0, w_k, w_k z_k, w_k (1 - z_k^2)
    float2* sw = sdy + I.nt;
    float2* swz = sw + I.nt;
    float2* sws = swz + I.nt;
    for (int k = threadIdx.x; k < qf2::kExpA + qf2::kExpB; k += blockDim.x) ta[k] = g.expt[k];
    for (int k = threadIdx.x; k < I.nt; k += blockDim.x) {
        const double y = g.y[I.t_off + k], w = g.wz[I.t_off + k];
        const qf2::f2 a = qf2::of(y - g.y[I.t_off]), b = qf2::of(w),
                      c = qf2::of(w * g.z[I.t_off + k]), d = qf2::of(w * g.s2[I.t_off + k]);
        sdy[k] = make_float2(a.h, a.l);
        sw[k] = make_float2(b.h, b.l);
        swz[k] = make_float2(c.h, c.l);
        sws[k] = make_float2(d.h, d.l);
    }
    __syncthreads();
    const int i0 = t.y * kTile, j0 = t.z * kTile;
    const double w = I.omega;
    const double iw2 = 1.0 / (w * w);
    const double pref = 8.0 * kPi * kPi / (w * w * w * w);
    const double y0 = g.y[I.t_off];
    const bool coll = (I.mode == QDSE_COLLOCATED);
    bool skip_tile;
    {
        const int i1 = min(i0 + kTile, I.n) - 1, j1 = min(j0 + kTile, I.n) - 1;
        const double pl = g.rsp[I.x_off + i0], ph = g.rsp[I.x_off + i1];
        const double ql = g.rsq[I.x_off + j0], qh = g.rsq[I.x_off + j1];
        const double gap = fmax(0.0, fmax(ql - ph, pl - qh));
        skip_tile = gap * gap * iw2 >= kSkipExponent;
    }
    const float* fta = reinterpret_cast<const float*>(ta);
    const float* ftb = reinterpret_cast<const float*>(tb);
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int li = e / kTile, lj = e % kTile;
        const int i = i0 + li, j = j0 + lj;
        qf2::f2 K0 = {0.f, 0.f}, KT = {0.f, 0.f}, K3 = {0.f, 0.f};
        if (!skip_tile && i < I.n && j < I.n) {
            const double P = g.sp[I.x_off + i], rP = g.rsp[I.x_off + i];
            const double Q = g.sq[I.x_off + j], rQ = g.rsq[I.x_off + j];
            if ((rP - rQ) * (rP - rQ) * iw2 < kSkipExponent &&
                qf2::pair_entries(P, Q, rP, rQ, y0, iw2, pref, kAngularCut, I.nt,
                                  reinterpret_cast<const float*>(sdy),
                                  reinterpret_cast<const float*>(sw),
                                  reinterpret_cast<const float*>(swz),
                                  reinterpret_cast<const float*>(sws), fta, ftb, K0, KT, K3) &&
                !(coll && i == j)) {
                KT = qf2::div(KT, qf2::of(Q - P));
            }
        }
        const int o = li * (kTile + 1) + lj;
        tileK[0 * S + o] = make_float2(K0.h, K0.l);
        tileK[1 * S + o] = make_float2(KT.h, KT.l);
        tileK[2 * S + o] = make_float2(K3.h, K3.l);
    }
    __syncthreads();
    store_tile(I, g, t, Khi, Klo, true, [&](int p, int idx, float& h, float& l) {
        const float2 v = tileK[p * S + idx];
        h = v.x;
        l = v.y;
    });
}

// Row bands: the nonzero entries of row i are the j with (sqrt P_i - sqrt Q_j)^2 / w^2 below the
// skip threshold, a contiguous range because sqrt Q_j increases with j; stored widened to
// multiples of 4.  One thread per external point; the same FP64 test as the tiles.
__global__ void k_row_bands(const DevInst* __restrict__ inst, Grid g, int ntot) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ntot) return;
    const int b = g.row_inst[r];
    const DevInst I = inst[b];
    const double iw2 = 1.0 / (I.omega * I.omega);
    const double rP = g.rsp[r];
    const double* rq = g.rsq + I.x_off;
    auto inside = [&](int j) { return (rP - rq[j]) * (rP - rq[j]) * iw2 < kSkipExponent; };
    // the internal node nearest to p_i (binary search on sqrt Q), then the two ends of the
    // contiguous range around it (binary searches)
    int lo = 0, hi = I.n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (rq[mid] < rP) lo = mid;
        else hi = mid;
    }
    const int c = (fabs(rq[lo] - rP) <= fabs(rq[hi] - rP)) ? lo : hi;
    int jl = 0, jh = 0;
    if (inside(c)) {
        int a = -1, in = c;  // !inside(a) (or a = -1), inside(in)
        while (in - a > 1) {
            const int mid = (a + in) / 2;
            if (inside(mid)) in = mid;
            else a = mid;
        }
        jl = in;
        int in2 = c, out = I.n;  // inside(in2), !inside(out) (or out = n)
        while (out - in2 > 1) {
            const int mid = (in2 + out) / 2;
            if (inside(mid)) in2 = mid;
            else out = mid;
        }
        jh = in2 + 1;
        jl &= ~3;
        jh = (jh + 3) & ~3;
        if (jh > I.ld) jh = I.ld;
    }
    g.band[r] = make_int2(jl, jh);
    atomicAdd(g.nnz + b, (unsigned long long)(jh - jl));
}

cudaError_t launch_precompute(qdse_ctx* c, bool with_w) {
    cudaError_t e = cudaMemsetAsync(c->grid.nnz, 0, sizeof(unsigned long long) * c->n_inst,
                                    c->stream);
    if (e != cudaSuccess) return e;
    const size_t smem =
        ((with_w ? 2 : 1) * 3 * kTile * (kTile + 1) + 5 * (size_t)c->max_nt) * sizeof(double);
    prof_begin(c, PK_PRECOMPUTE);
    if (with_w) {
        k_precompute_tiles<true><<<c->n_tiles, 256, smem, c->stream>>>(
            c->d_inst, c->grid, c->d_tiles, c->d_Khi, c->d_Klo, c->d_Kwhi, c->d_Kwlo);
    } else if (c->precompute_kind == 1) {
        const size_t smem_f2 = (3 * kTile * (kTile + 1) + qf2::kExpA + qf2::kExpB + 4 * (size_t)c->max_nt) *
                               sizeof(float2);
        k_precompute_tiles_f2<<<c->n_tiles, 256, smem_f2, c->stream>>>(
            c->d_inst, c->grid, c->d_tiles, c->d_Khi, c->d_Klo);
    } else {
        k_precompute_tiles<false><<<c->n_tiles, 256, smem, c->stream>>>(
            c->d_inst, c->grid, c->d_tiles, c->d_Khi, c->d_Klo, nullptr, nullptr);
    }
    c->launches++;
    prof_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_PRECOMPUTE);
    k_row_bands<<<(c->n_total + 127) / 128, 128, 0, c->stream>>>(c->d_inst, c->grid, c->n_total);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t configure_precompute(int max_nt) {
    const size_t smem = (2 * 3 * kTile * (kTile + 1) + 5 * (size_t)max_nt) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_precompute_tiles<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_precompute_tiles<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const size_t smem_f2 =
        (3 * kTile * (kTile + 1) + qf2::kExpA + qf2::kExpB + 4 * (size_t)max_nt) * sizeof(float2);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_precompute_tiles_f2,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f2);
    return e;
}

// Host tables of qf2::exp_neg (exp(-a/4) and exp(-b/512) as (hi, lo) pairs of the FP64 values).
void exp_tables(std::vector<float2>& out) {
    out.resize(qf2::kExpA + qf2::kExpB);
    qf2::exp_tables(reinterpret_cast<float*>(out.data()));
}

}  // namespace qdse
