// k_precompute.cu -- angular kernel matrices of the Ball-Chiu gap equation.
//
// After the Dirac traces of Eqs. dsesys/dsesys2 every angular dependence of a sweep sits in three
// kernels that do not depend on A or B (Sec. II; the reduction is derived in the solver notes):
//   K_n(P_i, Q_j) = 8 pi^2/w^4 sum_k w_k exp(-k^2/w^2) g_n(P_i, Q_j, z_k),   n = 0, T, 3,
//   g_0 = 1,  g_T = 2 P Q (1 - z^2)/k^2,  g_3 = [3 x (P + Q) - 4 x^2 - 2 P Q]/k^2,
//   x = sqrt(P Q) z,  k^2 = (sqrt P - sqrt Q)^2 + 2 sqrt(P Q) (1 - z)  (no cancellation at z -> 1).
// The interaction strength D is factored out.  K_T only ever multiplies the difference quotients
// (F(q^2) - F(p^2))/(q^2 - p^2), so the pool stores K_T/(Q_j - P_i) and the sweep multiplies it
// by plain differences; on the collocated diagonal it stores K_T itself.
//
// Every entry is evaluated in FP64 and stored as a double-float pair (hi = fl32(K),
// lo = fl32(K - hi)): the FP32 sweeps read hi, the FP64 residual reads hi + lo (about 48 bits).
// Optionally the omega-derivatives dK_n/dw (factor -4/w + 2 k^2/w^3 on each term) are stored in a
// second pool for the adjoint's dF/dw.
#include "qdse_internal.h"

namespace qdse {

// Pairs with (sqrt P - sqrt Q)^2 / w^2 beyond this have every term below the smallest FP32
// subnormal once stored, so they are written as exact zeros without evaluating the sum.
constexpr double kSkipExponent = 130.0;

template <bool WITH_W>
__global__ void __launch_bounds__(128) k_precompute(const DevInst* __restrict__ inst, Grid g,
                                                    float* __restrict__ Khi,
                                                    float* __restrict__ Klo,
                                                    float* __restrict__ Kwhi,
                                                    float* __restrict__ Kwlo) {
    extern __shared__ double sm[];
    __shared__ int s_lo, s_hi;
    const int r = blockIdx.x;  // global external point
    const int b = g.row_inst[r];
    const DevInst I = inst[b];
    const int i = r - I.x_off;
    double* sy = sm;
    double* sz = sm + I.nt;
    double* ss = sm + 2 * I.nt;
    double* sw = sm + 3 * I.nt;
    for (int k = threadIdx.x; k < I.nt; k += blockDim.x) {
        sy[k] = g.y[I.t_off + k];
        sz[k] = g.z[I.t_off + k];
        ss[k] = g.s2[I.t_off + k];
        sw[k] = g.wz[I.t_off + k];
    }
    if (threadIdx.x == 0) {
        s_lo = I.ld;
        s_hi = -1;
    }
    __syncthreads();

    const double P = g.sp[r], rP = g.rsp[r];
    const double w = I.omega;
    const double iw2 = 1.0 / (w * w);
    const double pref = 8.0 * kPi * kPi / (w * w * w * w);
    const double fw0 = -4.0 / w, fw1 = 2.0 / (w * w * w);
    const long long plane = I.ld;  // planes of a row are adjacent
    const long long row = I.k_off + (long long)i * 3 * I.ld;

    for (int j = threadIdx.x; j < I.ld; j += blockDim.x) {
        double K0 = 0.0, KT = 0.0, K3 = 0.0, W0 = 0.0, WT = 0.0, W3 = 0.0;
        if (j < I.n) {
            const int gj = I.x_off + j;
            const double Q = g.sq[gj], rQ = g.rsq[gj];
            const double dd = (rP - rQ) * (rP - rQ);
            if (dd * iw2 < kSkipExponent) {
                atomicMin(&s_lo, j);
                atomicMax(&s_hi, j);
                const double c2 = 2.0 * rP * rQ, x0 = rP * rQ, PQ = P * Q, PpQ = P + Q;
                for (int k = 0; k < I.nt; ++k) {
                    const double k2 = dd + c2 * sy[k];
                    const double E = sw[k] * exp(-k2 * iw2);
                    const double rk = 1.0 / k2;
                    const double x = x0 * sz[k];
                    const double gT = 2.0 * PQ * ss[k] * rk;
                    const double g3 = (3.0 * x * PpQ - 4.0 * x * x - 2.0 * PQ) * rk;
                    K0 += E;
                    KT += E * gT;
                    K3 += E * g3;
                    if (WITH_W) {
                        const double f = fw0 + fw1 * k2;
                        W0 += E * f;
                        WT += E * f * gT;
                        W3 += E * f * g3;
                    }
                }
                const double dq = (I.mode == QDSE_COLLOCATED && i == j) ? 1.0 : 1.0 / (Q - P);
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
        const double kv[3] = {K0, KT, K3};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float hi = __double2float_rn(kv[p]);
            Khi[row + p * plane + j] = hi;
            Klo[row + p * plane + j] = __double2float_rn(kv[p] - (double)hi);
        }
        if (WITH_W) {
            const double wv[3] = {W0, WT, W3};
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const float hi = __double2float_rn(wv[p]);
                Kwhi[row + p * plane + j] = hi;
                Kwlo[row + p * plane + j] = __double2float_rn(wv[p] - (double)hi);
            }
        }
    }
    // the nonzero entries of a row are a contiguous range of j (|sqrt P - sqrt Q| grows
    // monotonically away from it); store it widened to multiples of 4
    __syncthreads();
    if (threadIdx.x == 0) {
        int lo = s_lo, hi = s_hi + 1;
        if (hi <= lo) {
            lo = 0;
            hi = 0;
        } else {
            lo &= ~3;
            hi = (hi + 3) & ~3;
            if (hi > I.ld) hi = I.ld;
        }
        g.band[r] = make_int2(lo, hi);
        atomicAdd(g.nnz + b, (unsigned long long)(hi - lo));
    }
}

cudaError_t launch_precompute(qdse_ctx* c, bool with_w) {
    const size_t smem = 4 * sizeof(double) * (size_t)c->max_nt;
    cudaError_t e0 = cudaMemsetAsync(c->grid.nnz, 0, sizeof(unsigned long long) * c->n_inst,
                                     c->stream);
    if (e0 != cudaSuccess) return e0;
    prof_begin(c, PK_PRECOMPUTE);
    if (with_w) {
        k_precompute<true><<<c->n_total, 128, smem, c->stream>>>(c->d_inst, c->grid, c->d_Khi,
                                                                 c->d_Klo, c->d_Kwhi, c->d_Kwlo);
    } else {
        k_precompute<false><<<c->n_total, 128, smem, c->stream>>>(c->d_inst, c->grid, c->d_Khi,
                                                                  c->d_Klo, nullptr, nullptr);
    }
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

}  // namespace qdse
