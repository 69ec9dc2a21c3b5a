// k_adjoint.cu -- transposed sweep, implicit-function adjoint and the chiral condensate.
//
// At a fixed point x* = F(x*) of the successive approximation (Eqs. jifen12, jifen122), a loss
// L(x*(theta)) has dL/dtheta = lambda^T dF/dtheta with lambda = J^T lambda + g, J = dF/dx at x*
// and g = dL/dx (implicit function theorem; no unrolled iterations are stored).  The transposed
// fixed point is solved by the same successive approximation, sweep by sweep.
//
// J^T w for a collocated grid is computed row by row (k_vjp_row_t; staggered grids: k_vjp_stag_rows
// and k_vjp_stag_assemble below): with alpha_i = w^A_i kappa D/P_i and
// beta_i = w^B_i kappa D, entry l collects
//   (own)     sum_j alpha_l dT^A_lj/dx_l + beta_l dT^B_lj/dx_l          (row l of the kernels)
//   (partner) sum_i alpha_i dT^A_il/dx_l + beta_i dT^B_il/dx_l          (column l = row l, since
//             K_0 and K_3 are symmetric and K_T/(Q - P) is antisymmetric on a collocated grid)
//   (diagonal) the removable-limit terms of rows l and of rows whose stencil contains l,
// where T^A, T^B are the pair terms of the forward sweep (k_sweep.cu) and x_l = A_l or B_l
// enters through a, b and e = W/(Q a^2 + b^2).  The pair j = l has no K_T part (it cancels).
// Everything here runs in FP64 on the double-float kernels.
#include <cfloat>

#include "qdse_internal.h"

namespace qdse {

__device__ double block_sum_a(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

__device__ double block_max_a(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? sh[threadIdx.x] : -DBL_MAX;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

// Per-point FP64 vectors at x*: a, b, u1, u2, u3 (e and its derivatives follow from them), the
// stencil quotients, and the weights alpha_i, beta_i of the current cotangent w.
// Stored in work.vec64 / dia64 (x* part, once) and work.dvec64 components 0, 1 (alpha, beta).
__global__ void k_vjp_prep(const DevInst* __restrict__ inst, const Ctl* __restrict__ ctl, Grid g,
                           Work w, const double* A, const double* B, const double* wA,
                           const double* wB, int ntot, int with_x) {
    const DevInst I = inst[blockIdx.x];
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
        if (with_x) {
            // values at internal node j (on a staggered grid the modified interpolation
            // between p_j and p_j+1, Eq. chazhiresult)
            const double wt = g.wt[gj];
            double a = A[gj], b = B[gj];
            if (wt != 0.0) {
                a += wt * (A[gj + 1] - a);
                b += wt * (B[gj + 1] - b);
            }
            const double Q = g.sq[gj];
            const double e = g.W[gj] / (Q * a * a + b * b);
            w.vec64[gj] = a;
            w.vec64[ntot + gj] = b;
            w.vec64[2 * ntot + gj] = e * b;
            w.vec64[3 * ntot + gj] = e * a;
            w.vec64[4 * ntot + gj] = e * a * Q;
            if (I.mode == QDSE_COLLOCATED) {
                const int s0 = I.x_off + g.sta[gj];
                const double* c = g.stc + 3 * (size_t)gj;
                w.dia64[gj] = c[0] * A[s0] + c[1] * A[s0 + 1] + c[2] * A[s0 + 2];
                w.dia64[ntot + gj] = c[0] * B[s0] + c[1] * B[s0 + 1] + c[2] * B[s0 + 2];
            }
        }
        const double scale = ctl->kappa * I.D;
        w.dvec64[gj] = wA[gj] * scale / g.sp[gj];
        w.dvec64[ntot + gj] = wB[gj] * scale;
    }
}

// (J^T w)_l for a collocated grid.  One warp per point l.  If add_g, writes J^T w + g.
// T = double: FP64 arithmetic on the double-float kernels (hi + lo); T = float: FP32 arithmetic on
// the FP32 kernels (hi), for the inner sweeps of the mixed-precision adjoint.  want_phase >= 0:
// only the instances in that phase (the mixed adjoint runs both kinds in one tick).
template <typename T>
__global__ void __launch_bounds__(256) k_vjp_row_t(const DevInst* __restrict__ inst,
                                                   const Ctl* __restrict__ ctl, Grid g, Work w,
                                                   const float* __restrict__ Khi,
                                                   const float* __restrict__ Klo,
                                                   const DevState* __restrict__ state,
                                                   double* JA, double* JB, const double* gA,
                                                   const double* gB, int ntot, int add_g,
                                                   int only_active, int want_phase) {
    constexpr bool LO = sizeof(T) == 8;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= ntot) return;
    const int bi = g.row_inst[r];
    if (only_active && state[bi].phase == PH_DONE) return;
    if (want_phase >= 0 && state[bi].phase != want_phase) return;
    const DevInst I = inst[bi];
    if (I.mode != QDSE_COLLOCATED) return;  // k_vjp_stag_rows / k_vjp_stag_assemble
    const int l = r - I.x_off;
    const int o = I.x_off;
    const KRow row(I, l);
    const double* va = w.vec64 + o;
    const double* vb = w.vec64 + ntot + o;
    const double* v1 = w.vec64 + 2 * ntot + o;
    const double* v2 = w.vec64 + 3 * ntot + o;
    const double* v3 = w.vec64 + 4 * ntot + o;
    const double* al = w.dvec64 + o;
    const double* be = w.dvec64 + ntot + o;
    const double* sp = g.sp + o;
    const T Pl = T(sp[l]), Al = T(va[l]), Bl = T(vb[l]);
    const T Q = T(g.sq[r]);
    const T d = Q * Al * Al + Bl * Bl;
    const T el = T(g.W[r]) / d;
    const T ca = T(-2) * el * Q * Al / d, cb = T(-2) * el * Bl / d;
    const T alpha_l = T(al[l]), beta_l = T(be[l]);
    T gAl = T(0), gBl = T(0);
    // K_lm vanishes outside row l's band, and K_ml = K_lm: both parts only need the band
    const int2 bd = g.band[r];
    const int mlo = bd.x, mhi = min(bd.y, I.n);
    if (ctl->vertex == QDSE_VERTEX_BC) {
        for (int m = mlo + lane; m < mhi; m += 32) {
            const long long o0 = row.off(0, m), o1 = row.off(1, m), o2 = row.off(2, m);
            const T K0 = LO ? T((double)Khi[o0] + (double)Klo[o0]) : T(Khi[o0]);
            T KT = LO ? T((double)Khi[o1] + (double)Klo[o1]) : T(Khi[o1]);
            const T K3 = LO ? T((double)Khi[o2] + (double)Klo[o2]) : T(Khi[o2]);
            if (m == l) KT = T(0);
            // own part: l plays the row index, m the partner
            const T u1 = T(v1[m]), u2 = T(v2[m]), u3 = T(v3[m]);
            gAl += alpha_l * (T(0.5) * (Pl * u2 + u3) * KT + T(0.5) * u2 * K3) +
                   beta_l * (-u1 * KT + T(1.5) * u1 * K0);
            gBl += alpha_l * (u1 * KT) + beta_l * (u2 * KT);
            // partner part: m plays the row index i, l the partner; K_ml = K_lm, KT_ml = -KT_lm
            const T KTi = -KT;
            const T Ai = T(va[m]), Bi = T(vb[m]), Pi = T(sp[m]), ai = T(al[m]), bi = T(be[m]);
            const T PpQ = Pi + Q;
            const T TAe = (-Bl * (Bl - Bi) - T(0.5) * PpQ * Al * (Al - Ai)) * KTi +
                          T(0.5) * Al * (Ai + Al) * K3;
            const T TBe = (Al * Bi - Bl * Ai) * KTi + T(1.5) * Bl * (Ai + Al) * K0;
            const T dTA_da = el * (T(-0.5) * PpQ * (T(2) * Al - Ai) * KTi + T(0.5) * (Ai + T(2) * Al) * K3);
            const T dTA_db = -el * (T(2) * Bl - Bi) * KTi;
            const T dTB_da = el * (Bi * KTi + T(1.5) * Bl * K0);
            const T dTB_db = el * (-Ai * KTi + T(1.5) * (Ai + Al) * K0);
            gAl += ai * (dTA_da + TAe * ca) + bi * (dTB_da + TBe * ca);
            gBl += ai * (dTA_db + TAe * cb) + bi * (dTB_db + TBe * cb);
        }
    } else {
        for (int m = mlo + lane; m < mhi; m += 32) {
            const long long o0 = row.off(0, m), o2 = row.off(2, m);
            const T K0 = LO ? T((double)Khi[o0] + (double)Klo[o0]) : T(Khi[o0]);
            const T K3 = LO ? T((double)Khi[o2] + (double)Klo[o2]) : T(Khi[o2]);
            const T ai = T(al[m]), bi = T(be[m]);
            gAl += ai * (el + Al * ca) * K3 + bi * T(3) * Bl * ca * K0;
            gBl += ai * Al * cb * K3 + bi * T(3) * (el + Bl * cb) * K0;
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        gAl += __shfl_xor_sync(0xffffffffu, gAl, s);
        gBl += __shfl_xor_sync(0xffffffffu, gBl, s);
    }
    if (lane != 0) return;
    if (ctl->vertex == QDSE_VERTEX_BC && I.mode == QDSE_COLLOCATED) {
        // removable-limit terms of every row i whose value depends on x_l
        const int i0 = l - 2 < 0 ? 0 : l - 2, i1 = l + 2 > I.n - 1 ? I.n - 1 : l + 2;
        for (int i = i0; i <= i1; ++i) {
            const long long od = KRow(I, i).off(1, i);
            const T KTd = LO ? T((double)Khi[od] + (double)Klo[od]) : T(Khi[od]);
            const T ai = T(al[i]), bi = T(be[i]);
            const T u1 = T(v1[i]), u2 = T(v2[i]), Pi = T(sp[i]);
            const T dA = T(w.dia64[o + i]), dB = T(w.dia64[ntot + o + i]);
            const int sidx = l - g.sta[o + i];
            if (sidx >= 0 && sidx <= 2) {
                const T c = T(g.stc[3 * (size_t)(o + i) + sidx]);
                gAl += KTd * (ai * (-Pi * u2 * c) + bi * (u1 * c));
                gBl += KTd * (ai * (-u1 * c) + bi * (-u2 * c));
            }
            if (i == l) {
                const T eA = T(-2) * el * Pi * Al / d, eB = T(-2) * el * Bl / d;
                gAl += KTd * (ai * (-Bl * eA * dB - Pi * (el + Al * eA) * dA) +
                              bi * (Bl * eA * dA - (el + Al * eA) * dB));
                gBl += KTd * (ai * (-(el + Bl * eB) * dB - Pi * Al * eB * dA) +
                              bi * ((el + Bl * eB) * dA - Al * eB * dB));
            }
        }
    }
    double outA = (double)gAl, outB = (double)gBl;
    if (add_g) {
        outA += gA[r];
        outB += gB[r];
    }
    JA[r] = outA;
    JB[r] = outB;
}

// J^T w on a staggered grid, where the internal nodes q_j are not the external points and the
// kernel matrices are not symmetric.  Row pass, one warp per external point i: the row's own
// derivatives (through A_i, B_i in the pair terms) go to JA_i, JB_i; the derivatives through the
// values a_j, b_j at internal node j (and e_j = W_j/(Q_j a_j^2 + b_j^2)) are summed over the rows
// into col[j] by FP64 atomic adds (so the last bits depend on the order of the adds).  The
// assembly pulls col back through the interpolation a_j = (1 - wt_j) A_j + wt_j A_j+1 (Eq.
// chazhiresult): point l receives (1 - wt_l) col[l] + wt_l-1 col[l - 1].
__global__ void __launch_bounds__(256) k_vjp_stag_rows(const DevInst* __restrict__ inst,
                                                       const Ctl* __restrict__ ctl, Grid g,
                                                       Work w, const float* __restrict__ Khi,
                                                       const float* __restrict__ Klo,
                                                       const DevState* __restrict__ state,
                                                       const double* A, const double* B,
                                                       double* JA, double* JB, double* col,
                                                       int ntot, int only_active) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= ntot) return;
    const int bi = g.row_inst[r];
    if (only_active && state[bi].phase == PH_DONE) return;
    const DevInst I = inst[bi];
    if (I.mode == QDSE_COLLOCATED) return;  // k_vjp_row_t
    const int i = r - I.x_off, o = I.x_off;
    const KRow row(I, i);
    const double Pi = g.sp[r], Ai = A[r], Bi = B[r];
    const double ai = w.dvec64[r], bi_ = w.dvec64[ntot + r];  // alpha_i, beta_i
    const bool bc = ctl->vertex == QDSE_VERTEX_BC;
    double oA = 0.0, oB = 0.0;
    const int2 bd = g.band[r];
    for (int j = bd.x + lane; j < min(bd.y, I.n); j += 32) {
        const int gj = o + j;
        const long long o0 = row.off(0, j), o1 = row.off(1, j), o2 = row.off(2, j);
        const double K0 = (double)Khi[o0] + (double)Klo[o0];
        const double KT = bc ? (double)Khi[o1] + (double)Klo[o1] : 0.0;
        const double K3 = (double)Khi[o2] + (double)Klo[o2];
        const double a = w.vec64[gj], b = w.vec64[ntot + gj];
        const double u1 = w.vec64[2 * ntot + gj], u2 = w.vec64[3 * ntot + gj],
                     u3 = w.vec64[4 * ntot + gj];
        const double Q = g.sq[gj], d = Q * a * a + b * b, e = g.W[gj] / d;
        const double ea = -2.0 * e * Q * a / d, eb = -2.0 * e * b / d;  // de/da, de/db
        double ca, cb;
        if (bc) {
            oA += ai * (0.5 * (Pi * u2 + u3) * KT + 0.5 * u2 * K3) +
                  bi_ * (-u1 * KT + 1.5 * u1 * K0);
            oB += ai * (u1 * KT) + bi_ * (u2 * KT);
            const double TAe = (-b * (b - Bi) - 0.5 * (Pi + Q) * a * (a - Ai)) * KT +
                               0.5 * a * (Ai + a) * K3;
            const double TBe = (a * Bi - b * Ai) * KT + 1.5 * b * (Ai + a) * K0;
            ca = ai * (e * (-0.5 * (Pi + Q) * (2.0 * a - Ai) * KT + 0.5 * (Ai + 2.0 * a) * K3) +
                       TAe * ea) +
                 bi_ * (e * (Bi * KT + 1.5 * b * K0) + TBe * ea);
            cb = ai * (e * (-(2.0 * b - Bi) * KT) + TAe * eb) +
                 bi_ * (e * (-Ai * KT + 1.5 * (Ai + a) * K0) + TBe * eb);
        } else {
            // rainbow: T^A = u2 K3, T^B = 3 u1 K0 (no dependence on A_i, B_i)
            ca = ai * (e + a * ea) * K3 + bi_ * 3.0 * b * ea * K0;
            cb = ai * a * eb * K3 + bi_ * 3.0 * (e + b * eb) * K0;
        }
        atomicAdd(col + gj, ca);
        atomicAdd(col + ntot + gj, cb);
    }
#pragma unroll
    for (int sft = 16; sft > 0; sft >>= 1) {
        oA += __shfl_xor_sync(0xffffffffu, oA, sft);
        oB += __shfl_xor_sync(0xffffffffu, oB, sft);
    }
    if (lane == 0) {
        JA[r] = oA;
        JB[r] = oB;
    }
}

__global__ void k_vjp_stag_assemble(const DevInst* __restrict__ inst, Grid g,
                                    const DevState* __restrict__ state, double* JA, double* JB,
                                    const double* col, const double* gA, const double* gB,
                                    int ntot, int add_g, int only_active) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ntot) return;
    const int bi = g.row_inst[r];
    if (only_active && state[bi].phase == PH_DONE) return;
    const DevInst I = inst[bi];
    if (I.mode == QDSE_COLLOCATED) return;
    const int l = r - I.x_off;
    const double wl = g.wt[r];
    double ja = JA[r] + (1.0 - wl) * col[r], jb = JB[r] + (1.0 - wl) * col[ntot + r];
    if (l > 0) {
        const double wp = g.wt[r - 1];
        ja += wp * col[r - 1];
        jb += wp * col[ntot + r - 1];
    }
    if (add_g) {
        ja += gA[r];
        jb += gB[r];
    }
    JA[r] = ja;
    JB[r] = jb;
}

// lambda <- (1 - alpha) lambda + alpha lambda_new with a max-norm relative stopping test.
__global__ void k_adjoint_update(const DevInst* __restrict__ inst, DevState* state,
                                 const Ctl* __restrict__ ctl, Grid g, Work w, int ntot,
                                 int* count, unsigned long long* ctr) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    DevState s = state[b];
    if (s.phase == PH_DONE) return;
    const DevInst I = inst[b];
    const double al = ctl->alpha;
    double dmax = 0.0, cmax = 0.0, bad = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int k = c * ntot + gj;
            const double ln = (1.0 - al) * w.lam[k] + al * w.lamn[k];
            dmax = fmax(dmax, fabs(ln));
            cmax = fmax(cmax, fabs(ln - w.lam[k]));
            if (!isfinite(ln)) bad = 1.0;
            w.lam[k] = ln;
        }
    }
    dmax = block_max_a(dmax, sh);
    cmax = block_max_a(cmax, sh);
    bad = block_max_a(bad, sh);
    // refresh alpha_i, beta_i for the next transposed sweep
    const double scale = ctl->kappa * I.D;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
        w.dvec64[gj] = w.lam[gj] * scale / g.sp[gj];
        w.dvec64[ntot + gj] = w.lam[ntot + gj] * scale;
    }
    if (threadIdx.x == 0) {
        if (ctr) {
            const unsigned long long n = (unsigned long long)I.n;
            atomicAdd(ctr + 1, 1ull);
            atomicAdd(ctr + 2, 24ull * g.nnz[blockIdx.x] + 96ull * n);
            atomicAdd(ctr + 3, n * n * (unsigned long long)I.nt);
        }
        s.iters += 1;
        s.change = dmax > 0.0 ? cmax / dmax : 0.0;
        if (bad != 0.0) {
            s.phase = PH_DONE;
            s.status = QDSE_ERR_NONFINITE;
        } else if (s.change <= ctl->tol) {
            s.phase = PH_DONE;
            s.status = QDSE_OK;
        } else if (s.iters >= ctl->max_iter) {
            s.phase = PH_DONE;
            s.status = QDSE_ERR_NOT_CONVERGED;
        }
        state[b] = s;
        if (s.phase != PH_DONE && count) atomicAdd(count, 1);
    }
}

// The mixed-precision adjoint: lambda = J^T lambda + g solved by defect correction, as the forward
// refinement solves x = F(x).  An instance alternates between
//   PH_RESID64   (FP64 transposed sweep on the double-float kernels): lamn = J^T lambda + g,
//                r = lamn - lambda; done when max|r| / max|lamn| <= tol (lambda <- lamn), else
//                delta = r and the inner solve starts;
//   PH_TANGENT32 (FP32 transposed sweep on the FP32 kernels): lamn = J32^T delta + r,
//                delta <- delta + alpha (lamn - delta) until its relative change is <= inner_tol
//                (or max_inner sweeps); then lambda <- lambda + delta and back to PH_RESID64.
// J32 differs from J by FP32 rounding (about 1e-7 relative), so each outer step shrinks the
// residual by about max(inner_tol / (1 - rho), 1e-6): the FP64 fixed point is reached after a few
// FP64 sweeps instead of one per Picard step.  The weights alpha_i, beta_i of the next sweep
// (dvec64) are those of lambda for PH_RESID64 and of delta for PH_TANGENT32.
__global__ void k_adjoint_update_mixed(const DevInst* __restrict__ inst, DevState* state,
                                       const Ctl* __restrict__ ctl, Grid g, Work w, int ntot,
                                       int* count, unsigned long long* ctr) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    DevState s = state[b];
    if (s.phase == PH_DONE) return;
    const DevInst I = inst[b];
    const double al = ctl->alpha;
    double dmax = 0.0, cmax = 0.0, bad = 0.0;
    const bool resid = (s.phase == PH_RESID64);
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int k = c * ntot + gj;
            const double ln = w.lamn[k];
            if (resid) {
                const double r = ln - w.lam[k];
                w.r64[k] = r;
                dmax = fmax(dmax, fabs(ln));
                cmax = fmax(cmax, fabs(r));
                if (!isfinite(ln)) bad = 1.0;
            } else {
                const double d = w.d64[k];
                const double dn = d + al * (ln - d);
                w.d64[k] = dn;
                dmax = fmax(dmax, fabs(dn));
                cmax = fmax(cmax, fabs(dn - d));
                if (!isfinite(dn)) bad = 1.0;
            }
        }
    }
    dmax = block_max_a(dmax, sh);
    cmax = block_max_a(cmax, sh);
    bad = block_max_a(bad, sh);
    const double change = dmax > 0.0 ? cmax / dmax : 0.0;
    int next = s.phase, status = s.status;
    bool done = false;
    if (bad != 0.0) {
        done = true;
        status = QDSE_ERR_NONFINITE;
    } else if (resid) {
        if (change <= ctl->tol) {
            done = true;
            status = QDSE_OK;
        } else {
            next = PH_TANGENT32;  // delta = r
        }
    } else if (change <= ctl->inner_tol || s.inner + 1 >= ctl->max_inner) {
        next = PH_RESID64;  // lambda += delta
    }
    if (!done && s.iters + 1 >= ctl->max_iter) {
        done = true;
        status = QDSE_ERR_NOT_CONVERGED;
    }
    // the new lambda or delta, and the weights of the next sweep
    const double scale = ctl->kappa * I.D;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int k = c * ntot + gj;
            if (resid) {
                if (done && status == QDSE_OK) w.lam[k] = w.lamn[k];
                else if (next == PH_TANGENT32) w.d64[k] = w.r64[k];
            } else if (next == PH_RESID64 || done) {
                w.lam[k] += w.d64[k];
            }
        }
        const double* src = (next == PH_TANGENT32) ? w.d64 : w.lam;
        w.dvec64[gj] = src[gj] * scale / g.sp[gj];
        w.dvec64[ntot + gj] = src[ntot + gj] * scale;
    }
    if (threadIdx.x == 0) {
        if (ctr) {
            const unsigned long long n = (unsigned long long)I.n;
            atomicAdd(ctr + (resid ? 1 : 0), 1ull);
            atomicAdd(ctr + 2, (resid ? 24ull : 12ull) * g.nnz[blockIdx.x] + 96ull * n);
            atomicAdd(ctr + 3, n * n * (unsigned long long)I.nt);
        }
        s.iters += 1;
        if (resid) {
            s.n64 += 1;
            s.change = change;
            s.inner = 0;
        } else {
            s.inner += 1;
            s.dnorm = change;
        }
        s.phase = done ? PH_DONE : next;
        s.status = status;
        state[b] = s;
        if (!done && count) atomicAdd(count, 1);
    }
}

// lambda = g to start; instances whose state is not a fixed point (relative residual rel above
// not_fixed; the implicit function theorem does not apply there) are marked finished at once.
__global__ void k_adjoint_init(const DevInst* __restrict__ inst, DevState* state, Work w,
                               const double* gA, const double* gB, int ntot, const double* rel,
                               double not_fixed, int phase0) {
    const DevInst I = inst[blockIdx.x];
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
        w.lam[gj] = gA[gj];
        w.lam[ntot + gj] = gB[gj];
    }
    if (threadIdx.x == 0) {
        DevState s{};
        s.phase = phase0;
        s.status = QDSE_ERR_NOT_CONVERGED;
        s.change = INFINITY;
        if (rel && !(rel[blockIdx.x] <= not_fixed)) s.phase = PH_DONE;
        state[blockIdx.x] = s;
    }
}

// g_params[4b + (0..3)] = (lambda_B . 1, lambda . Fh / D, lambda . Fw, 0) with Fh = F(x*) - x0
// and Fw = dF/domega at x*.
__global__ void k_adjoint_grads(const DevInst* __restrict__ inst,
                                const DevState* __restrict__ state, Work w, const double* Fh,
                                const double* Fw, double* gp, int* inst_status, int ntot) {
    __shared__ double sh[32];
    const DevInst I = inst[blockIdx.x];
    double sm = 0.0, sd = 0.0, sw = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
        const double la = w.lam[gj], lb = w.lam[ntot + gj];
        sm += lb;
        sd += la * Fh[gj] + lb * Fh[ntot + gj];
        sw += la * Fw[gj] + lb * Fw[ntot + gj];
    }
    sm = block_sum_a(sm, sh);
    sd = block_sum_a(sd, sh);
    sw = block_sum_a(sw, sh);
    if (threadIdx.x == 0) {
        gp[4 * blockIdx.x + 0] = sm;
        gp[4 * blockIdx.x + 1] = I.D != 0.0 ? sd / I.D : 0.0;
        gp[4 * blockIdx.x + 2] = sw;
        gp[4 * blockIdx.x + 3] = 0.0;
        if (inst_status) inst_status[blockIdx.x] = state[blockIdx.x].status;
    }
}

// ------------------------------------------------------------------------------------------------
// condensate  -<qbar q> = N_c/(4 pi^2) sum_j W_j b_j/(Q_j a_j^2 + b_j^2)
// ------------------------------------------------------------------------------------------------
__global__ void k_condensate(const DevInst* __restrict__ inst, Grid g, const double* A,
                             const double* B, double* out) {
    __shared__ double sh[32];
    const DevInst I = inst[blockIdx.x];
    double s = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
        const double wt = g.wt[gj];
        double a = A[gj], b = B[gj];
        if (wt != 0.0) {
            a += wt * (A[gj + 1] - a);
            b += wt * (B[gj + 1] - b);
        }
        s += g.W[gj] * b / (g.sq[gj] * a * a + b * b);
    }
    s = block_sum_a(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = 3.0 / (4.0 * kPi * kPi) * s;
}

// gA_l += cbar dC/dA_l, gB_l += cbar dC/dB_l, pulled back through the interpolation.
__global__ void k_condensate_vjp(const DevInst* __restrict__ inst, Grid g, const double* A,
                                 const double* B, const double* cbar, double* gA, double* gB) {
    const DevInst I = inst[blockIdx.x];
    const double c = cbar[blockIdx.x] * 3.0 / (4.0 * kPi * kPi);
    for (int l = threadIdx.x; l < I.n; l += blockDim.x) {
        double ga = 0.0, gb = 0.0;
        // internal nodes j = l (weight 1 - wt_l) and j = l - 1 (weight wt_{l-1}) use point l
        for (int j = l - 1; j <= l; ++j) {
            if (j < 0) continue;
            const int gj = I.x_off + j;
            const double wt = g.wt[gj];
            const double f = (j == l) ? (1.0 - wt) : wt;
            if (f == 0.0) continue;
            double a = A[gj], b = B[gj];
            if (wt != 0.0) {
                a += wt * (A[gj + 1] - a);
                b += wt * (B[gj + 1] - b);
            }
            const double Q = g.sq[gj], d = Q * a * a + b * b;
            ga += f * g.W[gj] * b * (-2.0 * Q * a) / (d * d);
            gb += f * g.W[gj] * (d - 2.0 * b * b) / (d * d);
        }
        gA[I.x_off + l] += c * ga;
        gB[I.x_off + l] += c * gb;
    }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
// The staggered instances' part of J^T w (row pass with column scatter, then the assembly).
static cudaError_t launch_vjp_staggered(qdse_ctx* c, const double* A, const double* B, double* JA,
                                        double* JB, int add_g, const double* gA, const double* gB,
                                        int only_active) {
    if (!c->any_staggered) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(c->work.col, 0, 2 * sizeof(double) * c->n_total, c->stream);
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_SWEEP);
    k_vjp_stag_rows<<<(c->n_total + 7) / 8, 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, c->d_state, A, B, JA, JB,
        c->work.col, c->n_total, only_active);
    c->launches++;
    prof_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_OTHER);
    k_vjp_stag_assemble<<<(c->n_total + 255) / 256, 256, 0, c->stream>>>(
        c->d_inst, c->grid, c->d_state, JA, JB, c->work.col, gA, gB, c->n_total, add_g,
        only_active);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_vjp(qdse_ctx* c, const double* A, const double* B, const double* wA,
                       const double* wB, double* JA, double* JB, int add_g, const double* gA,
                       const double* gB) {
    prof_begin(c, PK_OTHER);
    k_vjp_prep<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_ctl, c->grid, c->work, A, B, wA,
                                                 wB, c->n_total, 1);
    c->launches++;
    prof_end(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_SWEEP);
    k_vjp_row_t<double><<<(c->n_total + 7) / 8, 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, c->d_state, JA, JB, gA, gB,
        c->n_total, add_g, 0, -1);
    c->launches++;
    prof_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_vjp_staggered(c, A, B, JA, JB, add_g, gA, gB, 0);
}

cudaError_t launch_adjoint_init(qdse_ctx* c, double* lam, const double* gA, const double* gB,
                                const double* rel, double not_fixed, int phase0) {
    (void)lam;
    prof_begin(c, PK_OTHER);
    k_adjoint_init<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->work, gA, gB,
                                                     c->n_total, rel, not_fixed, phase0);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_prep(qdse_ctx* c, const double* A, const double* B) {
    prof_begin(c, PK_OTHER);
    k_vjp_prep<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_ctl, c->grid, c->work, A, B,
                                                 c->work.lam, c->work.lam + c->n_total,
                                                 c->n_total, 1);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_sweep(qdse_ctx* c, const double* A, const double* B, const double* gA,
                                 const double* gB) {
    prof_begin(c, PK_SWEEP);
    k_vjp_row_t<double><<<(c->n_total + 7) / 8, 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, c->d_state, c->work.lamn,
        c->work.lamn + c->n_total, gA, gB, c->n_total, 1, 1, -1);
    c->launches++;
    prof_end(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_vjp_staggered(c, A, B, c->work.lamn, c->work.lamn + c->n_total, 1, gA, gB, 1);
}

// One tick of the mixed-precision adjoint: the FP64 transposed sweep of the instances in
// PH_RESID64 (plus g), the FP32 one of those in PH_TANGENT32 (plus r), then the update.
cudaError_t launch_adjoint_mixed_tick(qdse_ctx* c, const double* gA, const double* gB,
                                      int* n_active) {
    const int blocks = (c->n_total + 7) / 8;
    prof_begin(c, PK_SWEEP);
    k_vjp_row_t<double><<<blocks, 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, c->d_state, c->work.lamn,
        c->work.lamn + c->n_total, gA, gB, c->n_total, 1, 1, PH_RESID64);
    c->launches++;
    prof_end(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_SWEEP);
    k_vjp_row_t<float><<<blocks, 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, c->d_state, c->work.lamn,
        c->work.lamn + c->n_total, c->work.r64, c->work.r64 + c->n_total, c->n_total, 1, 1,
        PH_TANGENT32);
    c->launches++;
    prof_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_UPDATE);
    k_adjoint_update_mixed<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->d_ctl,
                                                             c->grid, c->work, c->n_total,
                                                             n_active, c->d_sweeps);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_update(qdse_ctx* c, double* lam, const double* lam_new, int* n_active) {
    (void)lam;
    (void)lam_new;
    prof_begin(c, PK_UPDATE);
    k_adjoint_update<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->d_ctl, c->grid,
                                                       c->work, c->n_total, n_active,
                                                       c->d_sweeps);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_grads(qdse_ctx* c, const double* A, const double* B,
                                 const double* lam, const double* F, const double* Fw,
                                 double* g_params, int* inst_status) {
    (void)A;
    (void)B;
    (void)lam;
    prof_begin(c, PK_OTHER);
    k_adjoint_grads<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->work, F, Fw,
                                                      g_params, inst_status, c->n_total);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_condensate(qdse_ctx* c, const double* A, const double* B, double* out) {
    prof_begin(c, PK_OTHER);
    k_condensate<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->grid, A, B, out);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_condensate_vjp(qdse_ctx* c, const double* A, const double* B,
                                  const double* cbar, double* gA, double* gB) {
    prof_begin(c, PK_OTHER);
    k_condensate_vjp<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->grid, A, B, cbar, gA, gB);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

}  // namespace qdse
