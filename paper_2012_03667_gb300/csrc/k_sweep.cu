// k_sweep.cu -- successive-approximation sweeps of the Ball-Chiu gap equation and the per-instance
// solver state machine.
//
// One Jacobi sweep (Eq. jifen12 applied to Eqs. dsesys/dsesys2; every new A_i, B_i uses only the
// previous iterate) reads, for external point p_i,
//   A_i' = 1 + kappa D / P_i [ sum_j T^A_ij + diag^A_i ],   B_i' = m + kappa D [ sum_j T^B_ij + diag^B_i ]
// with kappa = C_F/(8 pi^3) and, for internal node q_j with a = A(q_j), b = B(q_j),
// e = W_j/(Q_j a^2 + b^2), u1 = e b, u2 = e a, u3 = e a Q_j (the BC vertex of Eq. 2 with
// Sigma_A = (A_i + a)/2 and the difference quotients folded into the stored K_T/(Q_j - P_i)):
//   T^A_ij = [-u1 (b - B_i) - (P_i u2 + u3)(a - A_i)/2] KT_ij + u2 (A_i + a)/2 K3_ij
//   T^B_ij = [ u1 (a - A_i) - u2 (b - B_i)] KT_ij + 3/2 u1 (A_i + a) K0_ij
// On a collocated grid the pair j = i contributes nothing to the KT terms (a = A_i, b = B_i) and
// the removable limit q^2 -> p^2 is added separately with the stencil quotients dA, dB at p_i:
//   diag^A_i = (-u1_i dB_i - P_i u2_i dA_i) K_T,ii,   diag^B_i = (u1_i dA_i - u2_i dB_i) K_T,ii.
// The bare (rainbow) vertex keeps only u2 K3 and 3 u1 K0.
//
// FP64 sweeps (residuals, FP64 Picard, tangents and the row maps of the C interface) take one
// warp per external point: lanes stride over j, read the three kernel entries and the per-node
// vectors, accumulate in registers and reduce by warp shuffles.  The FP32 sweeps of the batched
// solve take one warp per group of kRows consecutive points: the ring kernel (k_tick_ring, the
// default) streams a group's kernel block and node vectors through shared memory by bulk copies,
// the register kernel (k_tick) loads them straight from global memory; lanes own 4-column blocks
// and the group's row sums are reduced by one butterfly at the end of the group.
// The vectors (a, b, u1, u2, u3) are formed once per sweep per instance (O(N)) by the update
// kernel, which also owns the convergence test (Eq. jifenab2, relative form) and the phase
// transitions of the mixed-precision solve.
#include <algorithm>
#include <cfloat>

#include "qdse_internal.h"

namespace qdse {

// ------------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reductions for blockDim.x a multiple of 32 (<= 1024).  All threads get the result.
__device__ double block_max(double v, double* sh) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? sh[threadIdx.x] : -DBL_MAX;
    if (w == 0) r = warp_max(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The set of threads that updates one instance: a whole block (blockDim.x a multiple of 32).
struct BlockTeam {
    double* sh;  // at least 32 doubles of shared memory
    __device__ int tid() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ void sync() const { __syncthreads(); }
    __device__ double max(double v) const { return block_max(v, sh); }
    __device__ float maxf(float v) const {
        float* f = reinterpret_cast<float*>(sh);
        v = warp_maxf(v);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) f[threadIdx.x >> 5] = v;
        __syncthreads();
        const int l = threadIdx.x & 31;
        v = (l < (int)(blockDim.x >> 5)) ? f[l] : 0.f;
        return warp_maxf(v);  // every warp reduces the per-warp maxima itself
    }
    __device__ bool any(bool v) const { return __syncthreads_or(v) != 0; }
    // max of a and OR of f over the block in one exchange (every thread gets both)
    __device__ void maxf_or(float& a, int& f) const {
        a = warp_maxf(a);
        f = __any_sync(0xffffffffu, f != 0) ? 1 : 0;
        float* fs = reinterpret_cast<float*>(sh);
        int* is = reinterpret_cast<int*>(sh) + 32;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            fs[threadIdx.x >> 5] = a;
            is[threadIdx.x >> 5] = f;
        }
        __syncthreads();
        const int nw = blockDim.x >> 5;
        float m = fs[0];
        int o = is[0];
        for (int k = 1; k < nw; ++k) {
            m = fmaxf(m, fs[k]);
            o |= is[k];
        }
        __syncthreads();
        a = m;
        f = o;
    }
    // max of a and XOR of h over the block in one exchange (every thread gets both)
    __device__ void maxf_xor(float& a, unsigned long long& h) const {
        a = warp_maxf(a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
        float* fs = reinterpret_cast<float*>(sh);
        auto* hs = reinterpret_cast<unsigned long long*>(sh) + 8;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            fs[threadIdx.x >> 5] = a;
            hs[threadIdx.x >> 5] = h;
        }
        __syncthreads();
        const int nw = blockDim.x >> 5;
        float m = fs[0];
        unsigned long long x = hs[0];
        for (int k = 1; k < nw; ++k) {
            m = fmaxf(m, fs[k]);
            x ^= hs[k];
        }
        __syncthreads();
        a = m;
        h = x;
    }
    // XOR of v over the block (every thread gets it)
    __device__ unsigned long long xor_all(unsigned long long v) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
        auto* u = reinterpret_cast<unsigned long long*>(sh);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) u[threadIdx.x >> 5] = v;
        __syncthreads();
        v = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v ^= u[k];
        __syncthreads();
        return v;
    }
    __device__ bool leader() const { return threadIdx.x == 0; }
    // the leader's v to every thread
    __device__ int bcast(int v) const {
        __syncthreads();
        if (threadIdx.x == 0) reinterpret_cast<int*>(sh)[0] = v;
        __syncthreads();
        v = reinterpret_cast<const int*>(sh)[0];
        __syncthreads();
        return v;
    }
    // the leader's a and b to every thread (one exchange)
    __device__ void bcast2(int& a, int& b) const {
        __syncthreads();
        if (threadIdx.x == 0) {
            reinterpret_cast<int*>(sh)[0] = a;
            reinterpret_cast<int*>(sh)[1] = b;
        }
        __syncthreads();
        a = reinterpret_cast<const int*>(sh)[0];
        b = reinterpret_cast<const int*>(sh)[1];
        __syncthreads();
    }
};

// The set of threads that updates one instance inside the ring sweep: one warp (the one that swept
// the instance's last row group of the tick).
struct WarpTeam {
    __device__ int tid() const { return threadIdx.x & 31; }
    __device__ int size() const { return 32; }
    __device__ void sync() const { __syncwarp(); }
    __device__ double max(double v) const { return warp_max(v); }
    __device__ float maxf(float v) const { return warp_maxf(v); }
    __device__ bool any(bool v) const { return __any_sync(0xffffffffu, v) != 0; }
    __device__ bool leader() const { return (threadIdx.x & 31) == 0; }
    __device__ int bcast(int v) const { return __shfl_sync(0xffffffffu, v, 0); }
    __device__ void bcast2(int& a, int& b) const {
        a = __shfl_sync(0xffffffffu, a, 0);
        b = __shfl_sync(0xffffffffu, b, 0);
    }
    __device__ void maxf_or(float& a, int& f) const {
        a = warp_maxf(a);
        f = __any_sync(0xffffffffu, f != 0) ? 1 : 0;
    }
    __device__ void maxf_xor(float& a, unsigned long long& h) const {
        a = warp_maxf(a);
        h = xor_all(h);
    }
    __device__ unsigned long long xor_all(unsigned long long v) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
};

template <typename T, bool LO>
__device__ __forceinline__ T kload(const float* __restrict__ hi, const float* __restrict__ lo,
                                   long long idx) {
    if (LO) return (T)__ldg(hi + idx) + (T)__ldg(lo + idx);
    return (T)__ldg(hi + idx);
}

// R7 relative change of one point: |d| / max(|x_new|, floor); 0 when d == 0.
__device__ __forceinline__ double rel_change(double d, double xnew, double floor_) {
    d = fabs(d);
    if (d == 0.0) return 0.0;
    const double den = fmax(fabs(xnew), floor_);
    return den > 0.0 ? d / den : INFINITY;
}

// ------------------------------------------------------------------------------------------------
// per-node vectors
// ------------------------------------------------------------------------------------------------
// a, b at internal node j: on-grid (collocated) or the modified interpolation (staggered).
template <typename S>
__device__ __forceinline__ double at_q(const S* F, int gj, double wt) {
    double v = (double)F[gj];
    if (wt != 0.0) v += wt * ((double)F[gj + 1] - v);
    return v;
}

// Writes a, b, u1, u2, u3 for every node of instance I, and the diagonal stencil quotients
// dA/ds, dB/ds at p_i (collocated).  xa, xb: the iterate (FP32 or FP64 storage).  FP64 vectors
// put component c of node j at vec[c * vs + vb + j] (vs = ntot, vb = the instance's first global
// point); FP32 vectors use the blocked layout vpos(vb + j, c) with vb = the instance's first
// padded node (vs unused).
template <typename T>
__device__ __forceinline__ T& vslot(T* vec, int vs, int x, int c) {
    if constexpr (sizeof(T) == sizeof(float)) return vec[vpos(x, c)];
    else return vec[(size_t)c * vs + x];
}

template <typename S, typename T>
__device__ void prepare_vectors(const DevInst& I, const Grid& g, int ntot, const S* xa,
                                const S* xb, T* vec, int vs, int vb, T* dia, int tid = -1,
                                int nth = 0) {
    if (tid < 0) {
        tid = threadIdx.x;
        nth = blockDim.x;
    }
    for (int j = tid; j < I.n; j += nth) {
        const int gj = I.x_off + j;
        const double wt = g.wt[gj];
        const double a = at_q(xa, gj, wt), b = at_q(xb, gj, wt);
        const double Q = g.sq[gj];
        const double e = g.W[gj] / (Q * a * a + b * b);
        vslot(vec, vs, vb + j, 0) = (T)a;
        vslot(vec, vs, vb + j, 1) = (T)b;
        vslot(vec, vs, vb + j, 2) = (T)(e * b);
        vslot(vec, vs, vb + j, 3) = (T)(e * a);
        vslot(vec, vs, vb + j, 4) = (T)(e * a * Q);
        if (I.mode == QDSE_COLLOCATED) {
            const int s0 = I.x_off + g.sta[gj];
            const double* c = g.stc + 3 * (size_t)gj;
            dia[gj] = (T)(c[0] * (double)xa[s0] + c[1] * (double)xa[s0 + 1] +
                          c[2] * (double)xa[s0 + 2]);
            dia[ntot + gj] = (T)(c[0] * (double)xb[s0] + c[1] * (double)xb[s0 + 1] +
                                 c[2] * (double)xb[s0 + 2]);
        }
    }
}

// Tangent vectors at the iterate (xa, xb) in direction (va, vb):
// delta a, delta b, delta u1, delta u2, delta u3 and the stencil of the direction.
template <typename S, typename V, typename T>
__device__ void prepare_tangent(const DevInst& I, const Grid& g, int ntot, const S* xa,
                                const S* xb, const V* va, const V* vb, T* dvec, int vs, int vbase,
                                T* ddia, int tid = -1, int nth = 0) {
    if (tid < 0) {
        tid = threadIdx.x;
        nth = blockDim.x;
    }
    for (int j = tid; j < I.n; j += nth) {
        const int gj = I.x_off + j;
        const double wt = g.wt[gj];
        const double a = at_q(xa, gj, wt), b = at_q(xb, gj, wt);
        const double da = at_q(va, gj, wt), db = at_q(vb, gj, wt);
        const double Q = g.sq[gj];
        const double d = Q * a * a + b * b;
        const double e = g.W[gj] / d;
        const double de = -e * (2.0 * Q * a * da + 2.0 * b * db) / d;
        const double du2 = de * a + e * da;
        vslot(dvec, vs, vbase + j, 0) = (T)da;
        vslot(dvec, vs, vbase + j, 1) = (T)db;
        vslot(dvec, vs, vbase + j, 2) = (T)(de * b + e * db);
        vslot(dvec, vs, vbase + j, 3) = (T)du2;
        vslot(dvec, vs, vbase + j, 4) = (T)(du2 * Q);
        if (I.mode == QDSE_COLLOCATED) {
            const int s0 = I.x_off + g.sta[gj];
            const double* c = g.stc + 3 * (size_t)gj;
            ddia[gj] = (T)(c[0] * (double)va[s0] + c[1] * (double)va[s0 + 1] +
                           c[2] * (double)va[s0 + 2]);
            ddia[ntot + gj] = (T)(c[0] * (double)vb[s0] + c[1] * (double)vb[s0 + 1] +
                                  c[2] * (double)vb[s0 + 2]);
        }
    }
}

// FP32 node vectors from the FP32 iterate, computed in FP32 (they are stored in FP32): the same
// quantities as prepare_vectors, the stencil quotient in the difference form
// c0 (x0 - x1) + c2 (x2 - x1) (the coefficients of a derivative stencil sum to zero), which keeps
// FP32 accuracy where the iterate is flat.
__device__ void prepare_vectors32(const DevInst& I, const Grid& g, int ntot, const float* xa,
                                  const float* xb, float* vec, int vb, float* dia, int tid,
                                  int nth) {
    for (int j = tid; j < I.n; j += nth) {
        const int gj = I.x_off + j;
        const float wt = g.wt32[gj];
        float a = xa[gj], b = xb[gj];
        if (wt != 0.f) {
            a = fmaf(wt, xa[gj + 1] - a, a);
            b = fmaf(wt, xb[gj + 1] - b, b);
        }
        const float Q = g.sq32[gj];
        const float e = g.W32[gj] / fmaf(Q * a, a, b * b);
        const float ea = e * a;
        vec[vpos(vb + j, 0)] = a;
        vec[vpos(vb + j, 1)] = b;
        vec[vpos(vb + j, 2)] = e * b;
        vec[vpos(vb + j, 3)] = ea;
        vec[vpos(vb + j, 4)] = ea * Q;
        if (I.mode == QDSE_COLLOCATED) {
            const int s0 = I.x_off + g.sta[gj];
            const float* c = g.stc32 + 3 * (size_t)gj;
            dia[gj] = fmaf(c[0], xa[s0] - xa[s0 + 1], c[2] * (xa[s0 + 2] - xa[s0 + 1]));
            dia[ntot + gj] = fmaf(c[0], xb[s0] - xb[s0 + 1], c[2] * (xb[s0 + 2] - xb[s0 + 1]));
        }
    }
}

// R7 relative change in FP32: |d| / max(|x_new|, floor); 0 when d == 0.
__device__ __forceinline__ float rel_change32(float d, float xnew, float floor_) {
    d = fabsf(d);
    if (d == 0.f) return 0.f;
    const float den = fmaxf(fabsf(xnew), floor_);
    return den > 0.f ? d / den : INFINITY;
}

// ------------------------------------------------------------------------------------------------
// row kernels (one warp per external point)
// ------------------------------------------------------------------------------------------------
// Sums of one sweep row: sA, sB with F^A = 1 + kappa D sA / P_i, F^B = m + kappa D sB.
template <typename T, bool LO>
__device__ __forceinline__ void row_map(int lane, const DevInst& I, int i, T Pi, T Ai, T Bi,
                                        const T* __restrict__ vec, const T* __restrict__ dia,
                                        int ntot, const float* __restrict__ Khi,
                                        const float* __restrict__ Klo, int vertex, int jlo,
                                        int jhi, T& outA, T& outB) {
    if (jhi > I.n) jhi = I.n;
    const KRow row(I, i);
    const T* va = vec + I.x_off;
    const T* vb = vec + ntot + I.x_off;
    const T* v1 = vec + 2 * ntot + I.x_off;
    const T* v2 = vec + 3 * ntot + I.x_off;
    const T* v3 = vec + 4 * ntot + I.x_off;
    T sA = 0, sB = 0;
    if (vertex == QDSE_VERTEX_BC) {
#pragma unroll 4
        for (int j = jlo + lane; j < jhi; j += 32) {
            const T a = va[j], b = vb[j], u1 = v1[j], u2 = v2[j], u3 = v3[j];
            const T K0 = kload<T, LO>(Khi, Klo, row.off(0, j));
            const T KT = kload<T, LO>(Khi, Klo, row.off(1, j));
            const T K3 = kload<T, LO>(Khi, Klo, row.off(2, j));
            const T da = a - Ai, db = b - Bi, sa = Ai + a;
            const T cT = -u1 * db - (T)0.5 * (Pi * u2 + u3) * da;
            sA += cT * KT + (T)0.5 * u2 * sa * K3;
            sB += (u1 * da - u2 * db) * KT + (T)1.5 * u1 * sa * K0;
        }
    } else {
#pragma unroll 4
        for (int j = jlo + lane; j < jhi; j += 32) {
            const T K0 = kload<T, LO>(Khi, Klo, row.off(0, j));
            const T K3 = kload<T, LO>(Khi, Klo, row.off(2, j));
            sA += v2[j] * K3;
            sB += (T)3 * v1[j] * K0;
        }
    }
    sA = warp_sum(sA);
    sB = warp_sum(sB);
    if (vertex == QDSE_VERTEX_BC && I.mode == QDSE_COLLOCATED) {
        const T KTd = kload<T, LO>(Khi, Klo, row.off(1, i));
        const T dAi = dia[I.x_off + i], dBi = dia[ntot + I.x_off + i];
        sA += (-v1[i] * dBi - Pi * v2[i] * dAi) * KTd;
        sB += (v1[i] * dAi - v2[i] * dBi) * KTd;
    }
    outA = sA;
    outB = sB;
}

// Tangent of row_map in direction (dAi, dBi at p_i; dvec, ddia per node).
template <typename T, bool LO>
__device__ __forceinline__ void row_tangent(int lane, const DevInst& I, int i, T Pi, T Ai, T Bi,
                                            T dAi, T dBi, const T* __restrict__ vec,
                                            const T* __restrict__ dia,
                                            const T* __restrict__ dvec,
                                            const T* __restrict__ ddia, int ntot,
                                            const float* __restrict__ Khi,
                                            const float* __restrict__ Klo, int vertex, int jlo,
                                            int jhi, T& outA, T& outB) {
    if (jhi > I.n) jhi = I.n;
    const KRow row(I, i);
    const int o = I.x_off;
    T sA = 0, sB = 0;
    if (vertex == QDSE_VERTEX_BC) {
#pragma unroll 2
        for (int j = jlo + lane; j < jhi; j += 32) {
            const T a = vec[o + j], b = vec[ntot + o + j];
            const T u1 = vec[2 * ntot + o + j], u2 = vec[3 * ntot + o + j],
                    u3 = vec[4 * ntot + o + j];
            const T ea = dvec[o + j], eb = dvec[ntot + o + j];
            const T e1 = dvec[2 * ntot + o + j], e2 = dvec[3 * ntot + o + j],
                    e3 = dvec[4 * ntot + o + j];
            const T K0 = kload<T, LO>(Khi, Klo, row.off(0, j));
            const T KT = kload<T, LO>(Khi, Klo, row.off(1, j));
            const T K3 = kload<T, LO>(Khi, Klo, row.off(2, j));
            const T da = a - Ai, db = b - Bi, sa = Ai + a;
            const T dda = ea - dAi, ddb = eb - dBi, dsa = dAi + ea;
            const T t = Pi * u2 + u3, dt = Pi * e2 + e3;
            const T dcT = -e1 * db - u1 * ddb - (T)0.5 * (dt * da + t * dda);
            sA += dcT * KT + (T)0.5 * (e2 * sa + u2 * dsa) * K3;
            sB += (e1 * da + u1 * dda - e2 * db - u2 * ddb) * KT +
                  (T)1.5 * (e1 * sa + u1 * dsa) * K0;
        }
    } else {
#pragma unroll 4
        for (int j = jlo + lane; j < jhi; j += 32) {
            const T K0 = kload<T, LO>(Khi, Klo, row.off(0, j));
            const T K3 = kload<T, LO>(Khi, Klo, row.off(2, j));
            sA += dvec[3 * ntot + o + j] * K3;
            sB += (T)3 * dvec[2 * ntot + o + j] * K0;
        }
    }
    sA = warp_sum(sA);
    sB = warp_sum(sB);
    if (vertex == QDSE_VERTEX_BC && I.mode == QDSE_COLLOCATED) {
        const T KTd = kload<T, LO>(Khi, Klo, row.off(1, i));
        const int gi = o + i;
        const T u1 = vec[2 * ntot + gi], u2 = vec[3 * ntot + gi];
        const T e1 = dvec[2 * ntot + gi], e2 = dvec[3 * ntot + gi];
        const T dA = dia[gi], dB = dia[ntot + gi], edA = ddia[gi], edB = ddia[ntot + gi];
        sA += (-e1 * dB - u1 * edB - Pi * (e2 * dA + u2 * edA)) * KTd;
        sB += (e1 * dA + u1 * edA - e2 * dB - u2 * edB) * KTd;
    }
    outA = sA;
    outB = sB;
}

__device__ __forceinline__ float4 ld4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

// One (i, j) pair of the FP32 BC sweep (T^A_ij, T^B_ij of the header comment).
// h1 = 3/2 u1, h2 = 1/2 u2, h3 = 1/2 u3 are column factors, formed once per column by the caller.
__device__ __forceinline__ void pair32(float a, float b, float u1, float u2, float h1, float h2,
                                       float h3, float K0, float KT, float K3, float Ai, float Bi,
                                       float Pi, float& sA, float& sB) {
    const float da = a - Ai, db = b - Bi, sa = Ai + a;
    const float T = fmaf(Pi, h2, h3);                // (P_i u2 + u3) / 2
    const float cT = fmaf(-T, da, -u1 * db);
    sA = fmaf(cT, KT, fmaf(h2 * sa, K3, sA));
    sB = fmaf(fmaf(u1, da, -u2 * db), KT, fmaf(h1 * sa, K0, sB));
}

// The column factors of a lane's 4 columns.
struct Cols4 {
    float4 h1, h2, h3;
    __device__ Cols4(const float4& u1, const float4& u2, const float4& u3) {
        h1 = make_float4(1.5f * u1.x, 1.5f * u1.y, 1.5f * u1.z, 1.5f * u1.w);
        h2 = make_float4(0.5f * u2.x, 0.5f * u2.y, 0.5f * u2.z, 0.5f * u2.w);
        h3 = make_float4(0.5f * u3.x, 0.5f * u3.y, 0.5f * u3.z, 0.5f * u3.w);
    }
};

// Its tangent in direction (ea, eb, e1, e2, e3 at q_j; dAi, dBi at p_i).
__device__ __forceinline__ void tpair32(float a, float b, float u1, float u2, float u3, float ea,
                                        float eb, float e1, float e2, float e3, float K0,
                                        float KT, float K3, float Ai, float Bi, float dAi,
                                        float dBi, float Pi, float& sA, float& sB) {
    const float da = a - Ai, db = b - Bi, sa = Ai + a;
    const float dda = ea - dAi, ddb = eb - dBi, dsa = dAi + ea;
    const float t = fmaf(Pi, u2, u3), dt = fmaf(Pi, e2, e3);
    const float dcT = -e1 * db - u1 * ddb - 0.5f * (dt * da + t * dda);
    sA = fmaf(dcT, KT, fmaf(0.5f * fmaf(e2, sa, u2 * dsa), K3, sA));
    sB = fmaf(e1 * da + u1 * dda - e2 * db - u2 * ddb, KT, fmaf(1.5f * fmaf(e1, sa, u1 * dsa), K0, sB));
}

__device__ __forceinline__ float pick(const float4& v, int d) {
    return d == 0 ? v.x : (d == 1 ? v.y : (d == 2 ? v.z : v.w));
}

// Per-row state of the FP32 sweep of one row group (a lane's partial sums and the row constants).
struct Rows32 {
    float Ai[kRows], Bi[kRows], Pi[kRows], dAi[kRows], dBi[kRows], sA[kRows], sB[kRows];
    float qA[kRows], qB[kRows], eqA[kRows], eqB[kRows];
    double Pd[kRows];
};

template <bool TAN>
__device__ __forceinline__ void rows32_load(Rows32& R, const GroupDesc& d, const Grid& g,
                                            const Work& w, int ntot, int collocated) {
    const int o = d.x_off + d.i0;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        R.sA[r] = 0.f;
        R.sB[r] = 0.f;
        const bool v = r < d.nr;
        R.Pd[r] = v ? g.sp[o + r] : 1.0;
        R.Ai[r] = v ? w.x32[o + r] : 0.f;
        R.Bi[r] = v ? w.x32[ntot + o + r] : 0.f;
        R.Pi[r] = v ? g.sp32[o + r] : 0.f;
        R.dAi[r] = (v && TAN) ? w.d32[o + r] : 0.f;
        R.dBi[r] = (v && TAN) ? w.d32[ntot + o + r] : 0.f;
        R.qA[r] = (v && collocated) ? w.dia32[o + r] : 0.f;
        R.qB[r] = (v && collocated) ? w.dia32[ntot + o + r] : 0.f;
        R.eqA[r] = (v && collocated && TAN) ? w.ddia32[o + r] : 0.f;
        R.eqB[r] = (v && collocated && TAN) ? w.ddia32[ntot + o + r] : 0.f;
    }
}

// The pair sums of one lane's 4 consecutive columns for every row of the group.  K(r, p) returns
// the 4 kernel entries of plane p of row r at those columns; dd0 = i0 - (first column) locates
// the diagonal (the removable limit of row i0 + r sits at column offset dd0 + r when in [0, 4)).
template <bool TAN, typename KLoad>
__device__ __forceinline__ void rows32_chunk(Rows32& R, const KLoad& K, int nr, int dd0, bool bc,
                                             int collocated, const float4& a, const float4& b,
                                             const float4& u1, const float4& u2,
                                             const float4& u3, const float4& ea,
                                             const float4& eb, const float4& e1,
                                             const float4& e2, const float4& e3) {
    const Cols4 H(u1, u2, u3);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (r < nr) {
            const float4 K0 = K(r, 0), K3 = K(r, 2);
            if (bc) {
                const float4 KT = K(r, 1);
                if (!TAN) {
                    pair32(a.x, b.x, u1.x, u2.x, H.h1.x, H.h2.x, H.h3.x, K0.x, KT.x, K3.x, R.Ai[r], R.Bi[r], R.Pi[r], R.sA[r], R.sB[r]);
                    pair32(a.y, b.y, u1.y, u2.y, H.h1.y, H.h2.y, H.h3.y, K0.y, KT.y, K3.y, R.Ai[r], R.Bi[r], R.Pi[r], R.sA[r], R.sB[r]);
                    pair32(a.z, b.z, u1.z, u2.z, H.h1.z, H.h2.z, H.h3.z, K0.z, KT.z, K3.z, R.Ai[r], R.Bi[r], R.Pi[r], R.sA[r], R.sB[r]);
                    pair32(a.w, b.w, u1.w, u2.w, H.h1.w, H.h2.w, H.h3.w, K0.w, KT.w, K3.w, R.Ai[r], R.Bi[r], R.Pi[r], R.sA[r], R.sB[r]);
                } else {
                    tpair32(a.x, b.x, u1.x, u2.x, u3.x, ea.x, eb.x, e1.x, e2.x, e3.x, K0.x, KT.x, K3.x, R.Ai[r], R.Bi[r], R.dAi[r], R.dBi[r], R.Pi[r], R.sA[r], R.sB[r]);
                    tpair32(a.y, b.y, u1.y, u2.y, u3.y, ea.y, eb.y, e1.y, e2.y, e3.y, K0.y, KT.y, K3.y, R.Ai[r], R.Bi[r], R.dAi[r], R.dBi[r], R.Pi[r], R.sA[r], R.sB[r]);
                    tpair32(a.z, b.z, u1.z, u2.z, u3.z, ea.z, eb.z, e1.z, e2.z, e3.z, K0.z, KT.z, K3.z, R.Ai[r], R.Bi[r], R.dAi[r], R.dBi[r], R.Pi[r], R.sA[r], R.sB[r]);
                    tpair32(a.w, b.w, u1.w, u2.w, u3.w, ea.w, eb.w, e1.w, e2.w, e3.w, K0.w, KT.w, K3.w, R.Ai[r], R.Bi[r], R.dAi[r], R.dBi[r], R.Pi[r], R.sA[r], R.sB[r]);
                }
                // removable limit q^2 -> p^2 of row i = i0 + r, by the lane holding column i
                const int dd = dd0 + r;
                if (collocated && dd >= 0 && dd < 4) {
                    const float KTd = pick(KT, dd), x1 = pick(u1, dd), x2 = pick(u2, dd);
                    if (!TAN) {
                        R.sA[r] += (-x1 * R.qB[r] - R.Pi[r] * x2 * R.qA[r]) * KTd;
                        R.sB[r] += (x1 * R.qA[r] - x2 * R.qB[r]) * KTd;
                    } else {
                        const float y1 = pick(e1, dd), y2 = pick(e2, dd);
                        R.sA[r] += (-y1 * R.qB[r] - x1 * R.eqB[r] -
                                    R.Pi[r] * (y2 * R.qA[r] + x2 * R.eqA[r])) * KTd;
                        R.sB[r] += (y1 * R.qA[r] + x1 * R.eqA[r] - y2 * R.qB[r] - x2 * R.eqB[r]) * KTd;
                    }
                }
            } else {
                const float4 p2 = TAN ? e2 : u2, p1 = TAN ? e1 : u1;
                R.sA[r] += p2.x * K3.x + p2.y * K3.y + p2.z * K3.z + p2.w * K3.w;
                R.sB[r] += 3.f * (p1.x * K0.x + p1.y * K0.y + p1.z * K0.z + p1.w * K0.w);
            }
        }
    }
}

// Warp totals of the group's 2 kRows sums and the stores of F(x) (or J delta) for its rows.
template <bool TAN>
__device__ __forceinline__ void rows32_store(const Rows32& R, const GroupDesc& d, int lane,
                                             const Work& w, int ntot, double scale, double m) {
    const float tot = group_totals(R.sA, R.sB, lane);
    const int qv = group_total_index(lane), r = qv % kRows;
    double P = 1.0;  // p_i^2 of the lane's row (unrolled select keeps R in registers)
#pragma unroll
    for (int k = 0; k < kRows; ++k)
        if (k == r) P = R.Pd[k];
    if (group_total_leader(lane) && r < d.nr) {
        const int gi = d.x_off + d.i0 + r;
        if (qv < kRows) {
            w.xn32[gi] = TAN ? (float)(scale * (double)tot / P)
                             : (float)(1.0 + scale * (double)tot / P);
        } else {
            w.xn32[ntot + gi] = TAN ? (float)(scale * (double)tot) : (float)(m + scale * (double)tot);
        }
    }
}

// FP32 sweep (or, with TAN, tangent sweep) of one row group: one warp, lanes over 4-node column
// chunks (16-byte loads) inside the union of the rows' nonzero bands.  The group descriptor carries
// every offset, so all loads of the group issue after a single round trip; the node vectors of a
// chunk serve every row; the removable-limit term of row i is added by the lane that holds column
// i (its kernel entry K_T,ii and node vectors are already in that lane's registers).
template <bool TAN>
__device__ __forceinline__ void group32(int lane, const GroupDesc& d, const Grid& g,
                                        const Work& w, int ntot, const float* __restrict__ Khi,
                                        int vertex, int collocated, double scale, double m) {
    Rows32 R;
    rows32_load<TAN>(R, d, g, w, ntot, collocated);
    const float* kb = Khi + d.kbase;
    const int nb = 3 * d.nr * 4;  // floats of one 4-column block
    const bool bc = (vertex == QDSE_VERTEX_BC);
    for (int c = d.jlo + 4 * lane; c < d.jhi; c += 128) {
        const float* vb = w.vec32 + vpos(d.v_off + c, 0);
        const float4 a = ld4(vb), b = ld4(vb + 4), u1 = ld4(vb + 8), u2 = ld4(vb + 12),
                     u3 = ld4(vb + 16);
        float4 ea, eb, e1, e2, e3;
        if (TAN) {
            const float* db_ = w.dvec32 + vpos(d.v_off + c, 0);
            ea = ld4(db_);
            eb = ld4(db_ + 4);
            e1 = ld4(db_ + 8);
            e2 = ld4(db_ + 12);
            e3 = ld4(db_ + 16);
        }
        const float* kc = kb + (long long)(c >> 2) * nb;
        const int sw = kswz(d.nr, c >> 2);
        auto K = [&](int r, int pl) { return ld4(kc + ((3 * r + pl) ^ sw) * 4); };
        rows32_chunk<TAN>(R, K, d.nr, d.i0 - c, bc, collocated, a, b, u1, u2, u3, ea, eb, e1, e2,
                          e3);
    }
    rows32_store<TAN>(R, d, lane, w, ntot, scale, m);
}

// One tick of the batched solve: every row group of every unfinished instance advances by the
// operation its instance's phase asks for (one warp per group).
// One row group of a tick; returns after its outputs are stored.
__device__ __forceinline__ void tick_group(const GroupDesc& d, int phase, int lane,
                                           const DevInst& I, const Ctl* __restrict__ ctl,
                                           const Grid& g, const Work& w,
                                           const float* __restrict__ Khi,
                                           const float* __restrict__ Klo, const double* A,
                                           const double* B, int ntot) {
    const int vertex = ctl->vertex;
    const int collocated = (I.mode == QDSE_COLLOCATED) && vertex == QDSE_VERTEX_BC;
    const double scale = ctl->kappa * I.D;
    if (phase == PH_PICARD32) {
        group32<false>(lane, d, g, w, ntot, Khi, vertex, collocated, scale, I.m);
    } else if (phase == PH_TANGENT32) {
        group32<true>(lane, d, g, w, ntot, Khi, vertex, collocated, scale, I.m);
    } else {  // PH_RESID64 or PH_PICARD64 on the precomputed double-float kernels
        for (int rr = 0; rr < d.nr; ++rr) {
            const int i = d.i0 + rr, r = I.x_off + i;
            const int2 bd = g.band[r];
            double sA, sB;
            row_map<double, true>(lane, I, i, g.sp[r], A[r], B[r], w.vec64, w.dia64, ntot, Khi,
                                  Klo, vertex, bd.x, bd.y, sA, sB);
            if (lane == 0) {
                w.xn64[r] = 1.0 + scale * sA / g.sp[r];
                w.xn64[ntot + r] = I.m + scale * sB;
            }
        }
    }
}

// Copy every instance's parameters into its row groups' descriptors (after each upload): the
// FP32 sweep's scale kappa D and mass m.
__global__ void k_group_params(const DevInst* __restrict__ inst, Grid g, int ngroups, int nslabs,
                               double kappa) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ngroups) {
        const DevInst I = inst[g.gdesc[t].b];
        g.gdesc[t].mode = I.mode;
        g.gdesc[t].sc32 = (float)(kappa * I.D);
        g.gdesc[t].m32 = (float)I.m;
    }
    if (t < nslabs) {
        const DevInst I = inst[g.slabs[t].b];
        g.slabs[t].sc32 = (float)(kappa * I.D);
        g.slabs[t].m32 = (float)I.m;
    }
}

// Narrow every group's column range to the union of its rows' nonzero bands.
__global__ void k_group_bands(const DevInst* __restrict__ inst, Grid g, int ngroups) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ngroups) return;
    GroupDesc d = g.gdesc[t];
    int lo = 1 << 30, hi = 0;
    for (int r = 0; r < d.nr; ++r) {
        const int2 bd = g.band[d.x_off + d.i0 + r];
        lo = min(lo, bd.x);
        hi = max(hi, bd.y);
    }
    if (hi <= lo) lo = hi = 0;
    g.gdesc[t].jlo = lo;
    g.gdesc[t].jhi = hi;
    // ... and the same band in the group's slab record
    const int lg = d.i0 / kRows;  // the group's index in its instance
    const int s_off = inst[d.b].s_off;
    g.slabs[s_off + lg / kSlabGroups].band[lg % kSlabGroups] = make_int2(lo, hi);
    // the narrow tail: every full group after the last full group wider than kNarrowCols
    if (d.nr == kRows && hi - lo > kNarrowCols) atomicMax(g.nfirst + d.b, lg + 1);
}

// ------------------------------------------------------------------------------------------------
// FP64 on-the-fly sweep: the (j, theta) double sum of Eqs. dsesys/dsesys2 for every point, with
// exp() per term and no precomputed kernel matrices.  One warp per external point; lanes stride
// over the internal nodes of the row's band, the j with (sqrt P - sqrt Q)^2 / w^2 < kOtfSkip:
// every term of any other pair carries exp(-k^2/w^2) <= e^-70 and moves the row's sum by less than
// 1e-20 of it (the argument of the precompute's bands).  Inside a pair the exponents k^2/w^2 grow
// with the node index, and the angular sum stops once a term's exponent exceeds the first one's by
// kOtfCut.  With k^2 = P + Q - 2x, 3x(P + Q) - 4x^2 - 2PQ = 3x k^2 - 2PQ(1 - z^2), so
// g_3 = 3x - g_T exactly: each term adds E = w_k exp(-k^2/w^2) against 1 and z and E(1 - z^2)/k^2
// (one exp and one division), and K_3 = 3 sqrt(PQ) sum(E z) - K_T has no cancellation near the
// diagonal (where the numerator of g_3 vanishes with k^2).
// ------------------------------------------------------------------------------------------------
constexpr double kOtfSkip = 70.0;
constexpr double kOtfCut = 60.0;

// The band [jlo, jhi) of row P (sqrt P = rP) over the increasing internal nodes rq[0..n).
__device__ __forceinline__ int2 otf_band(double rP, const double* __restrict__ rq, int n,
                                         double iw2) {
    auto inside = [&](int j) { return (rP - rq[j]) * (rP - rq[j]) * iw2 < kOtfSkip; };
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (rq[mid] < rP) lo = mid;
        else hi = mid;
    }
    const int c = (fabs(rq[lo] - rP) <= fabs(rq[hi] - rP)) ? lo : hi;
    if (!inside(c)) return make_int2(0, 0);
    int a = -1, in = c;
    while (in - a > 1) {
        const int mid = (a + in) / 2;
        if (inside(mid)) in = mid;
        else a = mid;
    }
    int in2 = c, out = n;
    while (out - in2 > 1) {
        const int mid = (in2 + out) / 2;
        if (inside(mid)) in2 = mid;
        else out = mid;
    }
    return make_int2(in, in2 + 1);
}

constexpr int kOtfRowsPerBlock = 8;

__global__ void __launch_bounds__(32 * kOtfRowsPerBlock)
    k_sweep_otf(const DevInst* __restrict__ inst, const DevState* __restrict__ state,
                const Ctl* __restrict__ ctl, Grid g, Work w, const double* __restrict__ A,
                const double* __restrict__ B, double* __restrict__ FA, double* __restrict__ FB,
                int ntot, int only_active) {
    const int r = blockIdx.x * kOtfRowsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= ntot) return;
    const int b = g.row_inst[r];
    if (only_active && state[b].phase == PH_DONE) return;
    const DevInst I = inst[b];
    const int i = r - I.x_off;
    const double* __restrict__ ty = g.y + I.t_off;
    const double* __restrict__ tz = g.z + I.t_off;
    const double* __restrict__ ts = g.s2 + I.t_off;
    const double* __restrict__ tw = g.wz + I.t_off;
    const int vertex = ctl->vertex;
    const double P = g.sp[r], rP = g.rsp[r];
    const double Ai = A[r], Bi = B[r];
    const double iw2 = 1.0 / (I.omega * I.omega);
    const double pref = 8.0 * kPi * kPi * I.D / (I.omega * I.omega * I.omega * I.omega);
    const int2 band = otf_band(rP, g.rsq + I.x_off, I.n, iw2);
    double sA = 0.0, sB = 0.0;
    for (int j = band.x + lane; j < band.y; j += 32) {
        const int gj = I.x_off + j;
        const double a = w.vec64[gj], bq = w.vec64[ntot + gj];
        const double Q = g.sq[gj], rQ = g.rsq[gj];
        const double e = g.W[gj] / (Q * a * a + bq * bq);
        double qA, qB;  // difference quotients of Eq. 2
        if (I.mode == QDSE_COLLOCATED && j == i) {
            qA = w.dia64[gj];
            qB = w.dia64[ntot + gj];
        } else {
            qA = (a - Ai) / (Q - P);
            qB = (bq - Bi) / (Q - P);
        }
        const double SA = 0.5 * (Ai + a);
        const double dd = (rP - rQ) * (rP - rQ), c2 = 2.0 * rP * rQ, x0 = rP * rQ;
        const double PQ = P * Q, PpQ = P + Q;
        const double ex_last = (dd + c2 * ty[0]) * iw2 + kOtfCut;
        double S0 = 0.0, Sz = 0.0, St = 0.0;
        for (int k = 0; k < I.nt; ++k) {
            const double k2 = dd + c2 * ty[k];
            const double ex = k2 * iw2;
            if (ex > ex_last) break;
            const double E = tw[k] * exp(-ex);
            S0 += E;
            Sz = fma(E, tz[k], Sz);
            St += E * ts[k] / k2;
        }
        const double ST = 2.0 * PQ * St;
        const double S3 = 3.0 * x0 * Sz - ST;
        if (vertex == QDSE_VERTEX_BC) {
            sA += e * ((-bq * qB - 0.5 * PpQ * a * qA) * ST + a * SA * S3);
            sB += e * ((-a * qB + bq * qA) * ST + 3.0 * bq * SA * S0);
        } else {
            sA += e * a * S3;
            sB += 3.0 * e * bq * S0;
        }
    }
    sA = warp_sum(sA);
    sB = warp_sum(sB);
    if (lane == 0) {
        FA[r] = 1.0 + ctl->kappa * pref * sA / P;
        FB[r] = I.m + ctl->kappa * pref * sB;
    }
}

// ------------------------------------------------------------------------------------------------
// per-instance state machine
// ------------------------------------------------------------------------------------------------
__device__ void prepare_phase(int phase, const DevInst& I, const Grid& g, const Work& w, int ntot,
                              const double* A, const double* B, int tid = -1, int nth = 0) {
    if (phase == PH_PICARD32) {
        if (tid < 0) {
            tid = threadIdx.x;
            nth = blockDim.x;
        }
        prepare_vectors32(I, g, ntot, w.x32, w.x32 + ntot, w.vec32, I.v_off, w.dia32, tid, nth);
    } else if (phase == PH_RESID64 || phase == PH_PICARD64) {
        prepare_vectors<double, double>(I, g, ntot, A, B, w.vec64, ntot, I.x_off, w.dia64, tid,
                                        nth);
    } else if (phase == PH_TANGENT32) {
        prepare_tangent<float, float, float>(I, g, ntot, w.x32, w.x32 + ntot, w.d32,
                                             w.d32 + ntot, w.dvec32, w.nv, I.v_off, w.ddia32, tid,
                                             nth);
    }
}


// Set every instance to its first phase, convert the start to FP32 where needed and form the
// vectors of the first sweep.  One block per instance.
__global__ void k_init_state(const DevInst* __restrict__ inst, DevState* state,
                             const Ctl* __restrict__ ctl, Grid g, Work w, const double* A,
                             const double* B, int ntot, int phase0) {
    const int b = blockIdx.x;
    const DevInst I = inst[b];
    if (phase0 == PH_PICARD32) {
        for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
            const int gj = I.x_off + j;
            w.x32[gj] = (float)A[gj];
            w.x32[ntot + gj] = (float)B[gj];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DevState s;
        s.phase = phase0;
        s.iters = 0;
        s.inner = 0;
        s.status = QDSE_ERR_NOT_CONVERGED;
        s.change = INFINITY;
        s.dnorm = INFINITY;
        s.loc = (phase0 == PH_PICARD32) ? 1 : 0;
        s.n64 = 0;
        s.cbest = INFINITY;
        s.since = 0;
        s.stall_max = 0;
        s.nh = 0;
        s.href = 0;
        s.iref = 0;
        s.plen = 1;
        s.cyc_p = 0;
        s.cyc_at = 0;
        state[b] = s;
        w.ilist[atomicAdd(w.lcount + 0, 1)] = b;
        if (!(ctl->tc_picard && phase0 == PH_PICARD32)) {  // else the tensor-core sweep has it
            const int ng = (I.n + kRows - 1) / kRows;
            int n0 = ng, n1 = ng;  // row groups [n0, n1) go on the narrow list
            if (ctl->narrow_split && phase0 == PH_PICARD32) {
                n1 = I.n / kRows;
                n0 = min(g.nfirst[b], n1);
            }
            const int nn = n1 - n0;
            const int gb = atomicAdd(w.lcount + 3, ng - nn);
            const int nb = nn > 0 ? atomicAdd(w.lcount + 9, nn) : 0;
            for (int t = 0; t < ng; ++t) {
                if (t >= n0 && t < n1) w.nlist[nb + t - n0] = I.g_off + t;
                else w.glist[gb + (t < n0 ? t : t - nn)] = I.g_off + t;
            }
            if (ctl->slab_lists) {
                const int ns = (ng + kSlabGroups - 1) / kSlabGroups;
                const int sb = atomicAdd(w.lcount + 6, ns);
                for (int t = 0; t < ns; ++t) w.slist[sb + t] = I.s_off + t;
            }
        }
    }
    for (int t = threadIdx.x; t < (I.n + kRows - 1) / kRows; t += blockDim.x) g.gphase[I.g_off + t] = phase0;
    if (ctl->slab_lists)
        for (int t = threadIdx.x; t < (I.n + kRows * kSlabGroups - 1) / (kRows * kSlabGroups);
             t += blockDim.x)
            w.sphase[I.s_off + t] = phase0;
    if (threadIdx.x == 0) w.ticket[b] = 0;
    prepare_phase(phase0, I, g, w, ntot, A, B);
}

// Iterate hashes for the cycle stop.  Every point contributes the SplitMix64 finaliser (Steele, Lea,
// Flood 2014) of its bit pattern offset by its index; the contributions are combined by XOR, so
// the hash does not depend on the order of the block reduction.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long point_hash32(float a, float b, int j) {
    const unsigned long long v = ((unsigned long long)__float_as_uint(a) << 32) |
                                 (unsigned long long)__float_as_uint(b);
    return mix64(v + (unsigned long long)(j + 1) * 0x9E3779B97F4A7C15ull);
}
__device__ __forceinline__ unsigned long long point_hash64(double a, double b, int j) {
    const unsigned long long k = (unsigned long long)(2 * j + 1) * 0x9E3779B97F4A7C15ull;
    return mix64((unsigned long long)__double_as_longlong(a) + k) ^
           mix64((unsigned long long)__double_as_longlong(b) + k + 0x9E3779B97F4A7C15ull);
}

// Cycle stop of a successive-approximation phase (leader thread).  One sweep of the batched solve
// is a fixed function of the iterate alone (the sweep kernels and the update sum in a fixed
// order), so once the iterate equals an earlier one of the same phase, the phase repeats that
// stretch forever and can never reach the tolerance.  h is the hash of the new iterate; it is
// compared with the last kHashRing hashes of the phase and with a reference hash that moves
// forward after 1, 2, 4, ... hashes (Brent's cycle detection), so a cycle of any period p is found
// within about 2 max(p, start of the cycle) sweeps, and one of period <= kHashRing as soon as it
// has gone round once.  Equal hashes of different iterates (a 64-bit collision) would end an
// instance early; over a batch of thousands of instances and thousands of sweeps that chance is
// below 1e-10.  Returns the period found (0: none).
// match: bit k set when entry k of the ring (k < min(nh, kHashRing)) equals h.
__device__ __forceinline__ int cycle_check(DevState& s, unsigned long long h,
                                           unsigned long long* ring, unsigned match) {
    int period = 0;
    if (match) {
        // the first matching entry k holds hash number t with t % kHashRing == k, the latest such
        // t < nh
        const int k = __ffs(match) - 1;
        const int t = s.nh - 1 - ((s.nh - 1 - k) % kHashRing);
        period = s.nh - t;
    }
    if (!period && s.nh > 0 && h == s.href) period = s.nh - s.iref;
    ring[s.nh % kHashRing] = h;
    if (s.nh == 0 || s.nh - s.iref >= s.plen) {
        s.href = h;
        s.iref = s.nh;
        s.plen = (s.nh == 0) ? 1 : 2 * s.plen;
    }
    s.nh += 1;
    return period;
}

// Progress of a successive-approximation phase: the lowest relative change reached so far and the
// sweeps since it was set.  Returns true when the no-progress stop applies (stall_window > 0
// consecutive sweeps without a new lowest change).  Only the leader's copy of the state is
// stored, and every thread computes the same values.
__device__ __forceinline__ bool track_progress(DevState& s, const Ctl& C) {
    const float c = (float)s.change;
    if (c < s.cbest) {
        s.cbest = c;
        s.since = 0;
    } else {
        s.since += 1;
        if (s.since > s.stall_max) s.stall_max = s.since;
    }
    return C.stall_window > 0 && !C.never_converge && s.since >= C.stall_window;
}

// The block's hash of the new iterate (h: this thread's part) through cycle_check; true when the
// cycle stop applies.  Every thread of the team gets the same answer.
template <typename Team>
__device__ __forceinline__ bool picard_cycle_reduced(const Team& T, DevState& s, const Ctl& C,
                                                     unsigned long long h,
                                                     unsigned long long* ring);
template <typename Team>
__device__ __forceinline__ bool picard_cycle(const Team& T, DevState& s, const Ctl& C,
                                             unsigned long long h, unsigned long long* ring) {
    if (!C.stop_cycles || C.never_converge) return false;
    return picard_cycle_reduced(T, s, C, T.xor_all(h), ring);
}
// The same with the block's hash h already reduced.
template <typename Team>
__device__ __forceinline__ bool picard_cycle_reduced(const Team& T, DevState& s, const Ctl& C,
                                                     unsigned long long h,
                                                     unsigned long long* ring) {
    if (!C.stop_cycles || C.never_converge) return false;
    // the first warp compares the recorded hashes in parallel (one round of loads)
    unsigned match = 0;
    if (T.tid() < 32) {
        const int k = T.tid();
        const bool m = k < min(s.nh, kHashRing) && ring[k] == h;
        match = __ballot_sync(0xffffffffu, m);
    }
    int period = 0;
    if (T.leader()) {
        period = cycle_check(s, h, ring, match);
        if (period && !s.cyc_p) {
            s.cyc_p = period;
            s.cyc_at = s.iters;
        }
    } else {
        s.nh += 1;  // keep every thread's copy of the count in step (only the leader's is stored)
    }
    return T.bcast(period) != 0;
}

// Advance one instance after a tick.  One block (256 threads) per instance.
// Sweep outputs (xn32, xn64) are read with L2-coherent loads (they come from other SMs; this keeps
// the update correct even when it runs inside the kernel that wrote them).
// snew: NULL, or shared memory for 2 kMaxN floats: the block then keeps its points in registers
// (kUpdPts per thread) and builds the next FP32 sweep's node vectors from the new iterate there.
constexpr int kUpdThreads = 128;                                  // k_update's block
constexpr int kUpdPts = (kMaxN + kUpdThreads - 1) / kUpdThreads;  // points per thread

// prepare_vectors32 with the instance's new FP32 iterate in shared memory (xs[j], xs[kMaxN + j]):
// the same values, bitwise (the same operations on the same inputs).
__device__ void prepare_vectors32_shared(const DevInst& I, const Grid& g, int ntot,
                                         const float* xs, float* vec, int vb, float* dia, int tid,
                                         int nth) {
    const float* xa = xs;
    const float* xb = xs + kMaxN;
    for (int j = tid; j < I.n; j += nth) {
        const int gj = I.x_off + j;
        const float wt = g.wt32[gj];
        float a = xa[j], b = xb[j];
        if (wt != 0.f) {
            a = fmaf(wt, xa[j + 1] - a, a);
            b = fmaf(wt, xb[j + 1] - b, b);
        }
        const float Q = g.sq32[gj];
        const float e = g.W32[gj] / fmaf(Q * a, a, b * b);
        const float ea = e * a;
        vec[vpos(vb + j, 0)] = a;
        vec[vpos(vb + j, 1)] = b;
        vec[vpos(vb + j, 2)] = e * b;
        vec[vpos(vb + j, 3)] = ea;
        vec[vpos(vb + j, 4)] = ea * Q;
        if (I.mode == QDSE_COLLOCATED) {
            const int s0 = g.sta[gj];
            const float* c = g.stc32 + 3 * (size_t)gj;
            dia[gj] = fmaf(c[0], xa[s0] - xa[s0 + 1], c[2] * (xa[s0 + 2] - xa[s0 + 1]));
            dia[ntot + gj] = fmaf(c[0], xb[s0] - xb[s0 + 1], c[2] * (xb[s0 + 2] - xb[s0 + 1]));
        }
    }
}

template <typename Team>
__device__ void update_instance(const Team& T, int b, const DevInst* __restrict__ inst,
                                DevState* state, const Ctl* __restrict__ ctl, const Grid& g,
                                const Work& w, double* A, double* B, int ntot, int* count,
                                unsigned long long* ctr, int next_list, float* snew = nullptr) {
    DevState s = state[b];
    if (s.phase == PH_DONE) return;
    const DevInst I = inst[b];
    const Ctl C = *ctl;
    if (T.leader() && ctr) {
        // work counters of the sweep this update completes: instance-sweeps by precision,
        // algorithmic bytes (kernel rows + per-node vectors + own values and outputs) and
        // BC-kernel evaluations n_p * n_q * n_theta
        // (kernel bytes: only the nonzero band of every row has to be read)
        const unsigned long long n = (unsigned long long)I.n, nz = g.nnz[b];
        unsigned long long bytes;
        if (s.phase == PH_PICARD32) bytes = 12ull * nz + 36ull * n;
        else if (s.phase == PH_TANGENT32) bytes = 12ull * nz + 64ull * n;
        else if (C.precision == QDSE_FP64) bytes = 56ull * n;
        else bytes = 24ull * nz + 72ull * n;
        atomicAdd(ctr + ((s.phase == PH_PICARD32 || s.phase == PH_TANGENT32) ? 0 : 1), 1ull);
        atomicAdd(ctr + 2, bytes);
        atomicAdd(ctr + 3, n * n * (unsigned long long)I.nt);
    }
    const int o = I.x_off;
    int next = s.phase;
    bool done = false;
    int status = s.status;
    if (s.phase == PH_PICARD32) {
        // the grid constants the next sweep's node vectors need, into L1 while the change is
        // computed (one 128-byte line per thread)
        const int t = T.tid(), nl = (I.n + 31) / 32, nl3 = (3 * I.n + 31) / 32;
        const void* pf = nullptr;
        if (t < nl) pf = g.wt32 + o + 32 * t;
        else if (t < 2 * nl) pf = g.sq32 + o + 32 * (t - nl);
        else if (t < 3 * nl) pf = g.W32 + o + 32 * (t - 2 * nl);
        else if (t < 4 * nl) pf = g.sta + o + 32 * (t - 3 * nl);
        else if (t < 4 * nl + nl3) pf = g.stc32 + 3 * (size_t)o + 32 * (t - 4 * nl);
        if (pf) asm volatile("prefetch.global.L1 [%0];" ::"l"(pf));
    }

    bool fast32 = false;  // the FP32 iterate of this update is also in snew (see below)
    if (s.phase == PH_PICARD32) {
        // relaxed FP32 Picard step and its R7 relative change, in FP32 like the iterate
        const float al = (float)C.alpha, am = (float)(1.0 - C.alpha);
        bool bad;
        bool cycled;
        if (snew && I.n <= kUpdPts * T.size()) {
            // one pass of loads: every thread keeps its points in registers (the same arithmetic
            // as the loop form below, with two block exchanges instead of five)
            fast32 = true;
            float xa[kUpdPts], xb[kUpdPts], fa[kUpdPts], fb[kUpdPts];
            float bmax = 0.f;
            int badj = 0;
#pragma unroll
            for (int k = 0; k < kUpdPts; ++k) {
                const int j = T.tid() + k * T.size();
                if (j < I.n) {
                    const int gj = o + j;
                    xa[k] = w.x32[gj];
                    xb[k] = w.x32[ntot + gj];
                    fa[k] = fmaf(al, __ldcg(w.xn32 + gj), am * xa[k]);
                    fb[k] = fmaf(al, __ldcg(w.xn32 + ntot + gj), am * xb[k]);
                    bmax = fmaxf(bmax, fabsf(fb[k]));
                    badj |= (!isfinite(fa[k]) || !isfinite(fb[k])) ? 1 : 0;
                }
            }
            T.maxf_or(bmax, badj);
            bad = badj != 0;
            const float fl = 1e-12f * bmax;
            float ch = 0.f;
            unsigned long long hsh = 0;
#pragma unroll
            for (int k = 0; k < kUpdPts; ++k) {
                const int j = T.tid() + k * T.size();
                if (j < I.n) {
                    const int gj = o + j;
                    ch = fmaxf(ch, fmaxf(rel_change32(fa[k] - xa[k], fa[k], 0.f),
                                         rel_change32(fb[k] - xb[k], fb[k], fl)));
                    w.x32[gj] = fa[k];
                    w.x32[ntot + gj] = fb[k];
                    snew[j] = fa[k];
                    snew[kMaxN + j] = fb[k];
                    hsh ^= point_hash32(fa[k], fb[k], j);
                }
            }
            T.maxf_xor(ch, hsh);
            s.change = (double)ch;
            s.iters += 1;
            cycled = picard_cycle_reduced(T, s, C, hsh, w.hring + (size_t)b * kHashRing);
        } else {
            float bmax = 0.f;
            bool badj = false;
            for (int j = T.tid(); j < I.n; j += T.size()) {
                const int gj = o + j;
                const float fa = fmaf(al, __ldcg(w.xn32 + gj), am * w.x32[gj]);
                const float fb = fmaf(al, __ldcg(w.xn32 + ntot + gj), am * w.x32[ntot + gj]);
                bmax = fmaxf(bmax, fabsf(fb));
                badj = badj || !isfinite(fa) || !isfinite(fb);
            }
            bmax = T.maxf(bmax);
            bad = T.any(badj);
            const float fl = 1e-12f * bmax;
            float ch = 0.f;
            unsigned long long hsh = 0;
            for (int j = T.tid(); j < I.n; j += T.size()) {
                const int gj = o + j;
                const float xa = w.x32[gj], xb = w.x32[ntot + gj];
                const float fa = fmaf(al, __ldcg(w.xn32 + gj), am * xa);
                const float fb = fmaf(al, __ldcg(w.xn32 + ntot + gj), am * xb);
                ch = fmaxf(ch, fmaxf(rel_change32(fa - xa, fa, 0.f), rel_change32(fb - xb, fb, fl)));
                w.x32[gj] = fa;
                w.x32[ntot + gj] = fb;
                hsh ^= point_hash32(fa, fb, j);
            }
            s.change = (double)T.maxf(ch);
            s.iters += 1;
            cycled = picard_cycle(T, s, C, hsh, w.hring + (size_t)b * kHashRing);
        }
        const bool stalled = track_progress(s, C);
        // a change within the tolerance ends the phase even when the iterate repeated (a repeat
        // with change 0 is a fixed point, not a cycle)
        const bool fp32_done = C.final_phase == PH_PICARD32 && !C.never_converge &&
                               s.change <= C.tol;
        const bool to_fp64 = C.final_phase != PH_PICARD32 &&
                             (s.change <= C.sw_tol || s.iters >= C.max_fp32);
        if (bad) {
            done = true;
            status = QDSE_ERR_NONFINITE;
        } else if (fp32_done) {
            // FP32-only solves finish here; mixed solves always finish in FP64
            done = true;
            status = QDSE_OK;
        } else if (to_fp64) {
            next = PH_RESID64;  // hand the FP32 iterate to the FP64 refinement
        } else if (stalled || cycled) {
            done = true;
            status = QDSE_ERR_NOT_CONVERGED;
        }
    } else if (s.phase == PH_PICARD64 || s.phase == PH_RESID64) {
        // relaxed Picard step (or the residual of one) and its R7 relative change
        double bmax = 0.0, bad = 0.0;
        for (int j = T.tid(); j < I.n; j += T.size()) {
            const int gj = o + j;
            double fb = __ldcg(w.xn64 + ntot + gj);
            double fa = __ldcg(w.xn64 + gj);
            const double xb = B[gj], xa = A[gj];
            if (s.phase != PH_RESID64) {
                fa = (1.0 - C.alpha) * xa + C.alpha * fa;
                fb = (1.0 - C.alpha) * xb + C.alpha * fb;
            }
            bmax = fmax(bmax, fabs(fb));
            if (!isfinite(fa) || !isfinite(fb)) bad = 1.0;
        }
        bmax = T.max(bmax);
        bad = T.max(bad);
        const double fl = 1e-12 * bmax;
        double ch = 0.0;
        unsigned long long hsh = 0;
        for (int j = T.tid(); j < I.n; j += T.size()) {
            const int gj = o + j;
            double fa = __ldcg(w.xn64 + gj);
            double fb = __ldcg(w.xn64 + ntot + gj);
            const double xa = A[gj], xb = B[gj];
            if (s.phase != PH_RESID64) {
                fa = (1.0 - C.alpha) * xa + C.alpha * fa;
                fb = (1.0 - C.alpha) * xb + C.alpha * fb;
            }
            ch = fmax(ch, fmax(rel_change(fa - xa, fa, 0.0), rel_change(fb - xb, fb, fl)));
            if (s.phase == PH_PICARD64) {
                A[gj] = fa;
                B[gj] = fb;
                hsh ^= point_hash64(fa, fb, j);
            } else {  // residual: keep r = F(x) - x for the correction solve
                w.r64[gj] = fa - xa;
                w.r64[ntot + gj] = fb - xb;
            }
        }
        ch = T.max(ch);
        s.change = ch;
        s.iters += 1;
        s.n64 += 1;
        const bool stalled = (s.phase == PH_PICARD64) &&
                             (track_progress(s, C) ||
                              picard_cycle(T, s, C, hsh, w.hring + (size_t)b * kHashRing));
        if (bad != 0.0) {
            done = true;
            status = QDSE_ERR_NONFINITE;
        } else if (!C.never_converge && ch <= C.tol) {
            done = true;
            status = QDSE_OK;
        } else if (stalled) {
            done = true;
            status = QDSE_ERR_NOT_CONVERGED;
        }
        if (s.phase == PH_RESID64) {
            if (done && status == QDSE_OK) {
                // accept the FP64 Picard step from the refined iterate
                for (int j = T.tid(); j < I.n; j += T.size()) {
                    A[o + j] = __ldcg(w.xn64 + o + j);
                    B[o + j] = __ldcg(w.xn64 + ntot + o + j);
                }
            } else if (!done) {
                // start a correction solve delta = J delta + r at the current x
                for (int j = T.tid(); j < I.n; j += T.size()) {
                    const int gj = o + j;
                    w.d64[gj] = w.r64[gj];
                    w.d64[ntot + gj] = w.r64[ntot + gj];
                    w.d32[gj] = (float)w.r64[gj];
                    w.d32[ntot + gj] = (float)w.r64[ntot + gj];
                    w.x32[gj] = (float)A[gj];
                    w.x32[ntot + gj] = (float)B[gj];
                }
                T.sync();
                prepare_vectors32(I, g, ntot, w.x32, w.x32 + ntot, w.vec32, I.v_off, w.dia32,
                                  T.tid(), T.size());
                next = PH_TANGENT32;
                s.inner = 0;
            }
        }
    } else if (s.phase == PH_TANGENT32) {
        // delta <- delta + alpha (J delta + r - delta); relative change of delta (max norm)
        double dmax = 0.0, cmax = 0.0, bad = 0.0;
        for (int j = T.tid(); j < I.n; j += T.size()) {
            const int gj = o + j;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int k = c * ntot + gj;
                const double d = w.d64[k];
                const double dn = d + C.alpha * ((double)__ldcg(w.xn32 + k) + w.r64[k] - d);
                dmax = fmax(dmax, fabs(dn));
                cmax = fmax(cmax, fabs(dn - d));
                if (!isfinite(dn)) bad = 1.0;
                w.d64[k] = dn;
                w.d32[k] = (float)dn;
            }
        }
        dmax = T.max(dmax);
        cmax = T.max(cmax);
        bad = T.max(bad);
        s.iters += 1;
        s.inner += 1;
        s.dnorm = dmax > 0.0 ? cmax / dmax : 0.0;
        if (bad != 0.0) {
            done = true;
            status = QDSE_ERR_NONFINITE;
        } else if (s.dnorm <= C.inner_tol || s.inner >= C.max_inner) {
            for (int j = T.tid(); j < I.n; j += T.size()) {
                A[o + j] += w.d64[o + j];
                B[o + j] += w.d64[ntot + o + j];
            }
            next = PH_RESID64;
        }
    }
    if (!done && s.iters >= C.max_iter) {
        done = true;
        status = QDSE_ERR_NOT_CONVERGED;
    }
    T.sync();
    if (done) {
        next = PH_DONE;
    } else {
        if (next == PH_RESID64 && s.phase == PH_PICARD32) {
            for (int j = T.tid(); j < I.n; j += T.size()) {
                A[o + j] = (double)w.x32[o + j];
                B[o + j] = (double)w.x32[ntot + o + j];
            }
            T.sync();
        }
        if (fast32 && next == PH_PICARD32) {
            prepare_vectors32_shared(I, g, ntot, snew, w.vec32, I.v_off, w.dia32, T.tid(),
                                     T.size());
        } else if (next != PH_TANGENT32 || s.phase == PH_TANGENT32) {
            prepare_phase(next, I, g, w, ntot, A, B, T.tid(), T.size());
        } else {
            prepare_tangent<float, float, float>(I, g, ntot, w.x32, w.x32 + ntot, w.d32,
                                                 w.d32 + ntot, w.dvec32, w.nv, I.v_off,
                                                 w.ddia32, T.tid(), T.size());
        }
    }
    for (int t = T.tid(); t < (I.n + kRows - 1) / kRows; t += T.size()) g.gphase[I.g_off + t] = next;
    if (C.slab_lists)
        for (int t = T.tid(); t < (I.n + kRows * kSlabGroups - 1) / (kRows * kSlabGroups);
             t += T.size())
            w.sphase[I.s_off + t] = next;
    if (T.leader()) {
        if (next != s.phase) {  // a new phase starts its own progress and cycle records
            s.cbest = INFINITY;
            s.since = 0;
            s.nh = 0;
            s.iref = 0;
            s.plen = 1;
        }
        s.phase = next;
        s.status = status;
        if (next == PH_PICARD32) s.loc = 1;
        else if (next != PH_DONE) s.loc = 0;
        state[b] = s;
        if (!done) {
            if (count) atomicAdd(count, 1);
            // the instance stays on the active list of the next tick
            w.ilist[(size_t)next_list * w.n_inst + atomicAdd(w.lcount + next_list, 1)] = b;
        }
    }
    if (!done && !(C.tc_picard && next == PH_PICARD32)) {
        // ... and so do its row groups and slabs (FP32 Picard rows of a shared-kernel batch go
        // to the tensor-core sweep instead)
        const int ng = (I.n + kRows - 1) / kRows;
        const int ns = (ng + kSlabGroups - 1) / kSlabGroups;
        int n0 = ng, n1 = ng;  // row groups [n0, n1) go on the narrow list
        if (C.narrow_split && next == PH_PICARD32) {
            n1 = I.n / kRows;
            n0 = min(g.nfirst[b], n1);
        }
        const int nn = n1 - n0;
        int gb = 0, sb = 0;  // sb: the slab lists' base, or the narrow list's (never both)
        if (T.leader()) {  // both reservations in flight at once
            gb = atomicAdd(w.lcount + 3 + next_list, ng - nn);
            if (C.slab_lists) sb = atomicAdd(w.lcount + 6 + next_list, ns);
            else if (nn > 0) sb = atomicAdd(w.lcount + 9 + next_list, nn);
        }
        T.bcast2(gb, sb);
        for (int t = T.tid(); t < ng; t += T.size()) {
            if (t >= n0 && t < n1)
                w.nlist[(size_t)next_list * w.n_groups + sb + t - n0] = I.g_off + t;
            else
                w.glist[(size_t)next_list * w.n_groups + gb + (t < n0 ? t : t - nn)] = I.g_off + t;
        }
        if (C.slab_lists)
            for (int t = T.tid(); t < ns; t += T.size())
                w.slist[(size_t)next_list * w.n_slabs + sb + t] = I.s_off + t;
    }
    T.sync();
}

// Pool offset of column c0 (a multiple of 4) of a row group's block; columns [c0, c1) are one
// contiguous run of (c1 - c0) * 3 nr floats from here (kpos).
__device__ __forceinline__ long long group_run(const GroupDesc& d, int c0) {
    return d.kbase + (long long)(c0 >> 2) * 3 * d.nr * 4;
}

// Ask L2 to fetch the kernel block and node vectors of one row group ahead of its sweep over the
// union band [jlo, jhi): lane 0 the kernel run, lane 1 the node vectors (one run in the blocked
// layout).  Both are 16-byte aligned multiples of 16 bytes.
__device__ __forceinline__ void prefetch_group(const GroupDesc& d, int lane, const Work& w,
                                               const float* __restrict__ Khi) {
    if (d.jhi <= d.jlo || lane > 1) return;
    const float* p = lane == 0 ? Khi + group_run(d, d.jlo) : w.vec32 + vpos(d.v_off + d.jlo, 0);
    const int bytes = (d.jhi - d.jlo) * (lane == 0 ? 3 * d.nr : 5) * 4;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One tick of the batched solve: persistent warps walk the active row groups (list t % 3 built by
// the previous update) and advance each by the operation its instance's phase asks for.  Each warp
// keeps the group after next prefetching into L2 while it sweeps the current one, so the
// dependent loads of a group (descriptor, own values, kernel rows) meet L2 instead of DRAM.
__global__ void __launch_bounds__(256, kTickBlocksPerSM) k_tick(const DevInst* __restrict__ inst,
                                                 const Ctl* __restrict__ ctl, Grid g, Work w,
                                                 const float* __restrict__ Khi,
                                                 const float* __restrict__ Klo, const double* A,
                                                 const double* B, int ntot, int list) {
    const int lane = threadIdx.x & 31;
    const int nact = w.lcount[3 + list];
    const int* ids = w.glist + (size_t)list * w.n_groups;
    const int stride = gridDim.x * (blockDim.x >> 5);
    int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= nact) return;
    int id = ids[t];
    int id1 = (t + stride < nact) ? ids[t + stride] : -1;
    int id2 = (t + 2 * stride < nact) ? ids[t + 2 * stride] : -1;
    prefetch_group(g.gdesc[id], lane, w, Khi);
    if (id1 >= 0) prefetch_group(g.gdesc[id1], lane, w, Khi);
    while (t < nact) {
        const int t3 = t + 3 * stride;
        const int id3 = (t3 < nact) ? ids[t3] : -1;
        GroupDesc d2;
        if (id2 >= 0) d2 = g.gdesc[id2];
        const GroupDesc d = g.gdesc[id];
        const int phase = g.gphase[id];
        const DevInst I = inst[d.b];
        tick_group(d, phase, lane, I, ctl, g, w, Khi, Klo, A, B, ntot);
        if (id2 >= 0) prefetch_group(d2, lane, w, Khi);
        t += stride;
        id = id1;
        id1 = id2;
        id2 = id3;
    }
}

// ---------------------------------------------------------------------------------------------
// Ring sweep: the same tick, with each warp streaming its row groups through shared memory.
//
// Tiles.  A warp owns SLOTS tile slots; a tile is up to 128 columns of one group: the group's
// kernel block over those columns and the node vectors a, b, u1, u2, u3 there, one bulk copy each
// (cp.async.bulk, completion counted in bytes on the slot's mbarrier).  After the warp finishes a
// tile it refills the freed slot with the next tile of its group sequence, so the following
// tiles are in flight while it computes.
//
// Groups.  Everything else a group needs travels through small per-warp rings in shared memory,
// filled by small asynchronous copies (cp.async, tracked with commit/wait groups): when the
// copying side moves onto group k it reads k's descriptor and phase (requested two moves
// earlier), and requests the row constants of group k, the descriptor and phase of group k + 2
// (whose list id arrived two moves earlier) and the list id of group k + 4.  So it never waits on
// a global load, even when it moves over several short groups in a row, and the computing side
// finds a group's descriptor, phase and row constants in shared memory.  The removable-limit term of each row is added once per group by the lane that
// stores the row's total.  Groups in an FP64 phase take the global-memory path of tick_group and
// no slots.
constexpr int kTileCols = 128;                         // columns per tile (4 per lane)
constexpr int kVecOff = 3 * kRows * kTileCols;         // slot floats before the node vectors
constexpr int kTileFloats = (3 * kRows + 5) * kTileCols;
constexpr long long kRingWaitBudget = 2000000000LL;    // clock cycles (about 1 s)
static_assert((kTileFloats * sizeof(float)) % 16 == 0, "tile slots must stay 16-byte aligned");
static_assert(kRows == 4, "the queue's row-constant copies are laid out for groups of 4 rows");

struct RingDesc {         // a group's descriptor (with the instance parameters) and phase
    GroupDesc d;
    int phase, pad[3];
};
struct RingRows {         // a group's row constants
    float rc[6][kRows];   // per row: A_i, B_i (FP32 iterate), P_i, stencil dA/ds, dB/ds, K_T(i,i)
    float vd[2][4];       // u1, u2 at the group's own nodes (collocated removable limit)
    float tc[4][kRows];   // tangent: dA_i, dB_i, stencil of the direction (A, B)
    float td[2][4];       // tangent: du1, du2 at the group's own nodes
};
// One warp's rings when its copying side may run AHEAD groups ahead of its computing side (group
// ck): row constants of groups ck .. ck + AHEAD, descriptors up to ck + AHEAD + 2, list ids up to
// ck + AHEAD + 4.
template <int AHEAD>
struct RingQueue {
    static constexpr int kRc = AHEAD + 1, kDesc = AHEAD + 3, kId = AHEAD + 6;
    RingDesc desc[kDesc];
    RingRows rows[kRc];
    int id[kId];
    int pad[(4 - kId % 4) % 4];
};
static_assert(sizeof(RingDesc) % 16 == 0 && sizeof(RingRows) % 16 == 0 &&
                  sizeof(RingQueue<2>) % 16 == 0 && sizeof(RingQueue<3>) % 16 == 0 &&
                  sizeof(RingQueue<4>) % 16 == 0,
              "ring entries must stay 16-byte aligned");

// A ring shape: WARPS computing warps per block, SLOTS tile slots per warp, and the copying side at
// most AHEAD groups ahead of the computing side.
template <int WARPS, int SLOTS, int AHEAD>
struct RingCfg {
    static constexpr int kWarps = WARPS, kSlots = SLOTS, kAhead = AHEAD;
    using Queue = RingQueue<AHEAD>;
    static constexpr size_t kTileBytes = (size_t)WARPS * SLOTS * kTileFloats * sizeof(float);
    static constexpr size_t kBarBytes = (size_t)WARPS * SLOTS * 8;
    static constexpr size_t kSmem = kTileBytes + kBarBytes + (size_t)WARPS * sizeof(Queue);
    static_assert(kSmem <= 227 * 1024, "ring sweep shared memory");
    static_assert(kBarBytes % 16 == 0, "queue must start 16-byte aligned");
    static_assert(AHEAD >= 2 && AHEAD <= 4, "cp_wait covers 0 .. 4 pending groups");
};
using RingSweep = RingCfg<12, 2, 2>;  // the default shape
using RingDeep = RingCfg<8, 3, 3>;
using RingDeeper = RingCfg<6, 4, 4>;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool ring_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `parity` of a slot barrier; false once the budget has run out.
__device__ __forceinline__ bool ring_wait(uint32_t bar, uint32_t parity) {
    if (ring_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!ring_test(bar, parity)) {
        if (clock64() - t0 > kRingWaitBudget) return false;
    }
    return true;
}

// The same with an L2 policy: evict-first for data read once per sweep (the kernel pool), so the
// pool's stream does not displace the small per-point arrays every group reads; evict-last for
// the node vectors, which every group of an instance reads again.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_copy_hint(float* dst, const float* src, int bytes,
                                               uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
        "[%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"((uint32_t)bytes), "r"(bar), "l"(pol)
        : "memory");
}

// Small asynchronous global -> shared copies (4 or 16 bytes) and their commit / wait groups.
__device__ __forceinline__ void cp4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n (0 .. 4) of this thread's most recent copy groups are pending
__device__ __forceinline__ void cp_wait(int n) {
    if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else if (n == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (n == 3) asm volatile("cp.async.wait_group 3;" ::: "memory");
    else asm volatile("cp.async.wait_group 4;" ::: "memory");
}

// A narrow tile (at most 32 * 4 / SPLIT columns, typically the last of a band) of a full group's
// BC Picard sweep: the warp's lanes split the group's rows instead of leaving 32 - 32 / SPLIT lanes
// idle.  Lane l takes the 4-column block l % (32 / SPLIT) for rows (l / (32 / SPLIT)) * (4 /
// SPLIT) and on; its sums go back to those rows' accumulators by selects, so the warp totals at
// the end of the group are formed as for full tiles.
__device__ __forceinline__ float pick_row(const float* v, int r) {
    float x = v[0];
#pragma unroll
    for (int k = 1; k < kRows; ++k) x = (r == k) ? v[k] : x;
    return x;
}

template <int SPLIT>
__device__ __forceinline__ void narrow_tile32(Rows32& R, const float* sl, int c, int jhi, int lane) {
    constexpr int RPL = kRows / SPLIT, NB = 32 / SPLIT;
    const int rg = lane / NB, cb = lane % NB;
    const int col = c + 4 * cb;
    float tA[RPL], tB[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) tA[k] = tB[k] = 0.f;
    if (col < jhi) {
        const float* kb = sl + cb * (3 * kRows * 4);
        const float* vb = sl + kVecOff + cb * 20;
        auto V4 = [&](int comp) { return *reinterpret_cast<const float4*>(vb + 4 * comp); };
        const float4 a = V4(0), b = V4(1), u1 = V4(2), u2 = V4(3), u3 = V4(4);
        const int sw = ((col >> 2) >> 1) & 3;
        const Cols4 H(u1, u2, u3);
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
            const int r = rg * RPL + k;
            const float Ai = pick_row(R.Ai, r), Bi = pick_row(R.Bi, r), Pi = pick_row(R.Pi, r);
            auto K = [&](int pl) {
                return *reinterpret_cast<const float4*>(kb + ((3 * r + pl) ^ sw) * 4);
            };
            const float4 K0 = K(0), KT = K(1), K3 = K(2);
            pair32(a.x, b.x, u1.x, u2.x, H.h1.x, H.h2.x, H.h3.x, K0.x, KT.x, K3.x, Ai, Bi, Pi, tA[k], tB[k]);
            pair32(a.y, b.y, u1.y, u2.y, H.h1.y, H.h2.y, H.h3.y, K0.y, KT.y, K3.y, Ai, Bi, Pi, tA[k], tB[k]);
            pair32(a.z, b.z, u1.z, u2.z, H.h1.z, H.h2.z, H.h3.z, K0.z, KT.z, K3.z, Ai, Bi, Pi, tA[k], tB[k]);
            pair32(a.w, b.w, u1.w, u2.w, H.h1.w, H.h2.w, H.h3.w, K0.w, KT.w, K3.w, Ai, Bi, Pi, tA[k], tB[k]);
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
            const bool mine = (rg * RPL + k == r);
            R.sA[r] += mine ? tA[k] : 0.f;
            R.sB[r] += mine ? tB[k] : 0.f;
        }
    }
}

// The update of one instance by one warp inside the ring sweep (kept out of line: it runs once per
// instance and tick, and inlining it would cost the sweep registers).
__device__ __noinline__ void update_by_warp(int b, const DevInst* __restrict__ inst,
                                            DevState* state, const Ctl* __restrict__ ctl,
                                            const Grid& g, const Work& w, double* A, double* B,
                                            int ntot, int* count, unsigned long long* ctr,
                                            int next_list) {
    update_instance(WarpTeam{}, b, inst, state, ctl, g, w, A, B, ntot, count, ctr, next_list);
}

template <typename Cfg>
__global__ void __launch_bounds__(Cfg::kWarps * 32, 1)
    k_tick_ring(const DevInst* __restrict__ inst, DevState* state, const Ctl* __restrict__ ctl,
                Grid g, Work w, const float* __restrict__ Khi, const float* __restrict__ Klo,
                double* A, double* B, int ntot, int list, int* count, unsigned long long* ctr,
                int fused, int* err) {
    constexpr int S = Cfg::kSlots;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* ring = reinterpret_cast<float*>(smem) + (size_t)warp * S * kTileFloats;
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(smem + Cfg::kTileBytes) + warp * S;
    using Queue = typename Cfg::Queue;
    Queue& q = reinterpret_cast<Queue*>(smem + Cfg::kTileBytes + Cfg::kBarBytes)[warp];
    if (lane == 0) {
        for (int k = 0; k < S; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[k]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // The block takes every gridDim.x-th entry of the active group list (a sample of all the
    // instances, so blocks get even shares); its warps claim those groups one at a time (a shared
    // counter), each claiming four groups ahead of its copying side, so warps that drew short
    // groups take more of them.
    __shared__ int s_next;
    if (threadIdx.x == 0) s_next = 0;
    if (fused && blockIdx.x == 0 && threadIdx.x == 0) {
        // the lists of two ticks ahead start empty (read by the previous tick, appended to by
        // the next one)
        const int clr = (list + 2) % 3;
        w.lcount[clr] = 0;
        w.lcount[3 + clr] = 0;
        w.lcount[6 + clr] = 0;
        w.lcount[9 + clr] = 0;
    }
    __syncthreads();
    const int nact = w.lcount[3 + list];
    const int G = gridDim.x;
    const int cnt = (int)blockIdx.x < nact ? (nact - 1 - (int)blockIdx.x) / G + 1 : 0;
    const int* ids = w.glist + (size_t)list * w.n_groups + blockIdx.x;
    auto claim = [&]() -> int {
        int c = 0;
        if (lane == 0) c = atomicAdd(&s_next, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        return c < cnt ? c * G : -1;
    };
    int nmine = 1 << 30;  // groups this warp claimed: known once a claim fails
    // a bounded wait of an earlier launch of this solve ran out: leave the state as it is
    if (*reinterpret_cast<volatile const int*>(err)) return;
    const bool bc = (ctl->vertex == QDSE_VERTEX_BC);
    const int stall = ctl->stall_copies ? 16 : 0;
    const uint64_t pol = lane == 0 ? evict_first_policy() : evict_last_policy();

    // prologue: claim groups 0 .. 3 and fetch their list ids, then the descriptors and phases of
    // groups 0 and 1, as two commit groups (the first move waits for all but the most recent one)
    for (int k = 0; k < 4 && k < nmine; ++k) {
        const int c = claim();
        if (c < 0) nmine = k;
        else if (lane == 0) cp4(&q.id[k], ids + c);
    }
    if (nmine == 0) return;
    cp_commit();
    cp_wait(0);
    __syncwarp();
    if (lane < 10 && (lane / 5) < nmine) {
        const int k = lane / 5, part = lane % 5;
        const int id = q.id[k];
        if (part < 4) cp16(reinterpret_cast<int4*>(&q.desc[k].d) + part,
                           reinterpret_cast<const int4*>(g.gdesc + id) + part);
        else cp4(&q.desc[k].phase, g.gphase + id);
    }
    cp_commit();
    cp_commit();  // an empty group: the first move's wait for "all but one" covers the above

    // copying side: current group pk, its tiles from column pc while ptiles
    int pk = -1, pc = 0, pjhi = 0, pnr = 0, pvoff = 0;
    long long pkbase = 0;
    bool ptiles = false;
    unsigned issued = 0, consumed = 0;

    // one step of the copying side: issue one tile, or move onto the next group; false when
    // neither is possible (sequence done, or the queue would overrun the computing side at ck)
    auto produce = [&](int ck) -> bool {
        if (!ptiles) {
            const int k = pk + 1;
            if (k >= nmine || k - ck > Cfg::kAhead) return false;
            pk = k;
            cp_wait(1);  // group k's descriptor and phase, group k + 2's list id
            __syncwarp();
            const RingDesc& e = q.desc[k % Queue::kDesc];
            RingRows& rw = q.rows[k % Queue::kRc];
            const int ph = e.phase;
            const int o = e.d.x_off + e.d.i0, nr = e.d.nr, ib = e.d.v_off + e.d.i0;
            pjhi = e.d.jhi;
            pnr = nr;
            pvoff = e.d.v_off;
            pkbase = e.d.kbase;
            pc = e.d.jlo;
            ptiles = (ph == PH_PICARD32 || ph == PH_TANGENT32) && pjhi > pc;
            if (lane < 6 * kRows) {
                // row constants of group k
                const int arr = lane / kRows, r = lane % kRows;
                const float* src = arr == 0   ? w.x32 + o
                                   : arr == 1 ? w.x32 + ntot + o
                                   : arr == 2 ? g.sp32 + o
                                   : arr == 3 ? w.dia32 + o
                                   : arr == 4 ? w.dia32 + ntot + o
                                              : g.ktd + o;
                if (r < nr) cp4(&rw.rc[arr][r], src + r);
            } else if (lane < 6 * kRows + 2) {
                cp16(rw.vd[lane - 6 * kRows], w.vec32 + vpos(ib, 2 + lane - 6 * kRows));
            } else if (lane < 6 * kRows + 7) {
                // descriptor (4 x 16 bytes) and phase of group k + 2
                if (k + 2 < nmine) {
                    const int part = lane - 6 * kRows - 2, id = q.id[(k + 2) % Queue::kId];
                    RingDesc& n2 = q.desc[(k + 2) % Queue::kDesc];
                    if (part < 4) cp16(reinterpret_cast<int4*>(&n2.d) + part,
                                       reinterpret_cast<const int4*>(g.gdesc + id) + part);
                    else cp4(&n2.phase, g.gphase + id);
                }
            }
            if (ph == PH_TANGENT32) {
                if (lane < 4 * kRows) {
                    const int arr = lane / kRows, r = lane % kRows;
                    const float* src = arr == 0   ? w.d32 + o
                                       : arr == 1 ? w.d32 + ntot + o
                                       : arr == 2 ? w.ddia32 + o
                                                  : w.ddia32 + ntot + o;
                    if (r < nr) cp4(&rw.tc[arr][r], src + r);
                } else if (lane < 4 * kRows + 2) {
                    cp16(rw.td[lane - 4 * kRows], w.dvec32 + vpos(ib, 2 + lane - 4 * kRows));
                }
            }
            if (k + 4 < nmine) {
                const int c = claim();  // list id of group k + 4
                if (c < 0) nmine = k + 4;
                else if (lane == 0) cp4(&q.id[(k + 4) % Queue::kId], ids + c);
            }
            cp_commit();
            return true;
        }
        const int slot = issued % S;
        const uint32_t bar = smem_addr(&bars[slot]);
        const int cols = min(kTileCols, pjhi - pc);
        // the slot's previous tile was read by this warp (generic proxy) before these copies
        // (async proxy) overwrite it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"((uint32_t)(cols * (3 * pnr + 5) * 4 + stall))
                         : "memory");
        __syncwarp();
        if (lane < 2) {
            // lane 0: the kernel run, lane 1: the node vectors (one instruction for both)
            float* dst = ring + slot * kTileFloats + (lane ? kVecOff : 0);
            const float* src = lane ? w.vec32 + vpos(pvoff + pc, 0)
                                    : Khi + pkbase + (long long)(pc >> 2) * 3 * pnr * 4;
            bulk_copy_hint(dst, src, cols * (lane ? 5 : 3 * pnr) * 4, bar, pol);
        }
        ++issued;
        pc += kTileCols;
        if (pc >= pjhi) ptiles = false;
        return true;
    };
    auto fill = [&](int ck) {
        while (issued - consumed < (unsigned)S && produce(ck)) {
        }
    };

    // Once a group's outputs are stored, the warp counts it on its instance's ticket; the warp
    // whose count completes the instance (every other group's outputs are then stored and fenced)
    // advances the instance at once: the relaxed step, its convergence test and phase, and the
    // node vectors of the next sweep (the work of k_update in the two-launch form).
    const int next_list = (list + 1) % 3;
    auto group_done = [&](int b, int ngb) {
        if (!fused) return;  // k_update advances the instances after the sweep
        __threadfence();  // this warp's stores of the group's outputs, before its count
        __syncwarp();
        int last = 0;
        if (lane == 0) last = (atomicAdd(w.ticket + b, 1) == ngb - 1);
        if (__shfl_sync(0xffffffffu, last, 0)) {
            __threadfence();  // then the other groups' outputs (read through L2)
            update_by_warp(b, inst, state, ctl, g, w, A, B, ntot, count, ctr, next_list);
            if (lane == 0) w.ticket[b] = 0;
        }
    };

    // the lane that stores a total: value qv (rows' A sums, then B sums) of row rr
    const int qv = group_total_index(lane), rr = qv % kRows;
    const bool isB = qv >= kRows;
    bool ok = true;
    for (int ck = 0; ck < nmine; ++ck) {
        while (pk < ck && produce(ck)) {
        }
        fill(ck);
        cp_wait(pk - ck);  // group ck's row constants
        __syncwarp();
        const GroupDesc& d = q.desc[ck % Queue::kDesc].d;
        const int phase = q.desc[ck % Queue::kDesc].phase;
        const RingRows& e = q.rows[ck % Queue::kRc];
        if (phase != PH_PICARD32 && phase != PH_TANGENT32) {
            const GroupDesc dc = d;
            tick_group(dc, phase, lane, inst[dc.b], ctl, g, w, Khi, Klo, A, B, ntot);
            group_done(dc.b, dc.ng);
            continue;
        }
        const bool tan = (phase == PH_TANGENT32);
        const int collocated = (d.mode == QDSE_COLLOCATED) && bc;
        const int nr = d.nr, jlo = d.jlo, jhi = d.jhi, i0 = d.i0, o = d.x_off + i0;
        const bool full = !tan && bc && nr == kRows;
        Rows32 R;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            R.sA[r] = 0.f;
            R.sB[r] = 0.f;
            R.Ai[r] = e.rc[0][r];
            R.Bi[r] = e.rc[1][r];
            R.Pi[r] = e.rc[2][r];
            R.dAi[r] = tan ? e.tc[0][r] : 0.f;
            R.dBi[r] = tan ? e.tc[1][r] : 0.f;
        }
        for (int c = jlo; c < jhi; c += kTileCols) {
            const int slot = consumed % S;
            const bool got = ring_wait(smem_addr(&bars[slot]), (consumed / S) & 1);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            const int col = c + 4 * lane;
            const int wc = min(kTileCols, jhi - c);  // columns in this tile
            if (full && wc <= kTileCols / 4) {
                narrow_tile32<4>(R, ring + slot * kTileFloats, c, jhi, lane);
            } else if (full && wc <= kTileCols / 2) {
                narrow_tile32<2>(R, ring + slot * kTileFloats, c, jhi, lane);
            } else if (col < jhi) {
                const float* sl = ring + slot * kTileFloats;
                const float* vb = sl + kVecOff + lane * 20;
                auto V4 = [&](int comp) { return *reinterpret_cast<const float4*>(vb + 4 * comp); };
                const float4 a = V4(0), b = V4(1), u1 = V4(2), u2 = V4(3), u3 = V4(4);
                if (full) {
                    // the common case, specialised: Picard sweep of a full group, BC vertex
                    const float* kb = sl + lane * (3 * kRows * 4);
                    const int sw = ((col >> 2) >> 1) & 3;  // kswz of a full group
                    auto K = [&](int r, int pl) {
                        return *reinterpret_cast<const float4*>(kb + ((3 * r + pl) ^ sw) * 4);
                    };
                    rows32_chunk<false>(R, K, kRows, 0, true, 0, a, b, u1, u2, u3, a, a, a, a, a);
                } else {
                const float* kb = sl + lane * 3 * nr * 4;
                const int sw = kswz(nr, col >> 2);
                auto K = [&](int r, int pl) {
                    return *reinterpret_cast<const float4*>(kb + ((3 * r + pl) ^ sw) * 4);
                };
                if (tan) {
                    const float* db_ = w.dvec32 + vpos(d.v_off + col, 0);
                    const float4 ea = ld4(db_), eb = ld4(db_ + 4), e1 = ld4(db_ + 8),
                                 e2 = ld4(db_ + 12), e3 = ld4(db_ + 16);
                    rows32_chunk<true>(R, K, nr, 0, bc, 0, a, b, u1, u2, u3, ea, eb, e1, e2, e3);
                } else {
                    rows32_chunk<false>(R, K, nr, 0, bc, 0, a, b, u1, u2, u3, a, a, a, a, a);
                }
                }
            }
            __syncwarp();
            ++consumed;
            fill(ck);
        }
        if (!ok) break;
        float tot = group_totals(R.sA, R.sB, lane);
        if (group_total_leader(lane) && rr < nr) {
            const float Pl = e.rc[2][rr];
            if (collocated) {
                // removable limit q^2 -> p^2 of row i0 + rr (K_T(i,i) times the stencil
                // quotients and the node vectors at p_i)
                const float KTd = e.rc[5][rr], qA = e.rc[3][rr], qB = e.rc[4][rr];
                const float x1 = e.vd[0][rr], x2 = e.vd[1][rr];
                if (!tan) {
                    tot += isB ? (x1 * qA - x2 * qB) * KTd : (-x1 * qB - Pl * x2 * qA) * KTd;
                } else {
                    const float y1 = e.td[0][rr], y2 = e.td[1][rr];
                    const float eqA = e.tc[2][rr], eqB = e.tc[3][rr];
                    tot += isB ? (y1 * qA + x1 * eqA - y2 * qB - x2 * eqB) * KTd
                               : (-y1 * qB - x1 * eqB - Pl * (y2 * qA + x2 * eqA)) * KTd;
                }
            }
            const float sc = d.sc32;
            if (!isB) w.xn32[o + rr] = tan ? __fdividef(sc * tot, Pl) : 1.f + __fdividef(sc * tot, Pl);
            else w.xn32[ntot + o + rr] = tan ? sc * tot : d.m32 + sc * tot;
        }
        group_done(d.b, d.ng);
    }
    cp_wait(0);  // no small copy may land after the block has released its shared memory
    if (!ok) {
        // a tile copy never completed: report it, then wait (bounded) for this warp's copies
        // still in flight so that none lands after the block has released its shared memory
        if (lane == 0) atomicExch(err, 1);
        for (unsigned u = consumed; u < issued; ++u)
            ring_wait(smem_addr(&bars[u % S]), (u / S) & 1);
    }
}

// The row groups of the narrow list (Ctl::narrow_split): full groups of a Ball-Chiu FP32 Picard
// sweep whose band is at most kNarrowCols columns (high momenta, where (sqrt P - sqrt Q)^2 / w^2
// < 70 spans few nodes).  On the scan they are a third of the groups and hold 4% of the kernel
// entries, yet in the ring sweep each pays the whole per-group machinery (descriptor and row
// constant copies, a tile wait, the warp totals) for at most 128 pairs.  Here one warp takes four
// of them at once, eight lanes each, straight from global memory: lane cb of a group's eight
// holds the 4-column block cb for all four rows, the same per-(row, block) partial sums as the
// ring's narrow tile (narrow_tile32<4>), and the sums over the eight blocks run in the same tree,
// ((0 + 4) + (2 + 6)) + ((1 + 5) + (3 + 7)), as the ring's warp totals, whose other levels only
// add exact zeros.  So every output is bitwise the ring's.
__global__ void __launch_bounds__(256, 2) k_tick_narrow(Grid g, Work w,
                                                     const float* __restrict__ Khi, int ntot,
                                                     int list, const int* err) {
    // a bounded wait of this tick's ring sweep ran out: the solve stops
    if (*reinterpret_cast<volatile const int*>(err)) return;
    const int n = w.lcount[9 + list];
    const int* ids = w.nlist + (size_t)list * w.n_groups;
    const int lane = threadIdx.x & 31, seg = lane >> 3, cb = lane & 7;
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int k0 = 4 * wid; k0 < n; k0 += 4 * nw) {
        const int k = k0 + seg;
        const bool act = k < n;
        GroupDesc d{};
        if (act) d = g.gdesc[ids[k]];
        const int o = d.x_off + d.i0;
        float sA[kRows], sB[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) sA[r] = sB[r] = 0.f;
        const int col = d.jlo + 4 * cb;
        if (act && col < d.jhi) {
            const float* vb = w.vec32 + vpos(d.v_off + col, 0);
            const float4 a = ld4(vb), b = ld4(vb + 4), u1 = ld4(vb + 8), u2 = ld4(vb + 12),
                         u3 = ld4(vb + 16);
            const Cols4 H(u1, u2, u3);
            const float* kc = Khi + d.kbase + (long long)(col >> 2) * (3 * kRows * 4);
            const int sw = ((col >> 2) >> 1) & 3;  // kswz of a full group
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const float Ai = w.x32[o + r], Bi = w.x32[ntot + o + r], Pi = g.sp32[o + r];
                const float4 K0 = ld4(kc + ((3 * r + 0) ^ sw) * 4);
                const float4 KT = ld4(kc + ((3 * r + 1) ^ sw) * 4);
                const float4 K3 = ld4(kc + ((3 * r + 2) ^ sw) * 4);
                pair32(a.x, b.x, u1.x, u2.x, H.h1.x, H.h2.x, H.h3.x, K0.x, KT.x, K3.x, Ai, Bi, Pi, sA[r], sB[r]);
                pair32(a.y, b.y, u1.y, u2.y, H.h1.y, H.h2.y, H.h3.y, K0.y, KT.y, K3.y, Ai, Bi, Pi, sA[r], sB[r]);
                pair32(a.z, b.z, u1.z, u2.z, H.h1.z, H.h2.z, H.h3.z, K0.z, KT.z, K3.z, Ai, Bi, Pi, sA[r], sB[r]);
                pair32(a.w, b.w, u1.w, u2.w, H.h1.w, H.h2.w, H.h3.w, K0.w, KT.w, K3.w, Ai, Bi, Pi, sA[r], sB[r]);
            }
        }
        // totals over the group's eight lanes (shuffles stay inside each 8-lane segment)
#pragma unroll
        for (int m = 4; m >= 1; m >>= 1) {
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                sA[r] += __shfl_xor_sync(0xffffffffu, sA[r], m);
                sB[r] += __shfl_xor_sync(0xffffffffu, sB[r], m);
            }
        }
        if (act) {
            // lane cb stores value cb: A of row cb (cb < 4), else B of row cb - 4
            const int rr = cb & (kRows - 1);
            const bool isB = cb >= kRows;
            float tot = 0.f;
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (r == rr) tot = isB ? sB[r] : sA[r];
            const float Pl = g.sp32[o + rr];
            if (d.mode == QDSE_COLLOCATED) {
                // removable limit q^2 -> p^2 of row i0 + rr, as in the ring sweep
                const float KTd = g.ktd[o + rr], qA = w.dia32[o + rr], qB = w.dia32[ntot + o + rr];
                const float x1 = w.vec32[vpos(d.v_off + d.i0 + rr, 2)];
                const float x2 = w.vec32[vpos(d.v_off + d.i0 + rr, 3)];
                tot += isB ? (x1 * qA - x2 * qB) * KTd : (-x1 * qB - Pl * x2 * qA) * KTd;
            }
            const float sc = d.sc32;
            if (!isB) w.xn32[o + rr] = 1.f + __fdividef(sc * tot, Pl);
            else w.xn32[ntot + o + rr] = d.m32 + sc * tot;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Slab sweep: the tick of k_tick_ring with the bookkeeping done per slab instead of per row group.
// A slab is up to kSlabGroups consecutive row groups (32 rows) of one instance, so its groups share
// the instance's phase, grid mode, vectors and parameters.  Per slab a warp
//   - reads the slab's 128-byte record (instance offsets, parameters, every group's band) and its
//     phase, requested two slabs ahead by small asynchronous copies (cp.async), like the list id
//     of the slab after that;
//   - finds the row constants of its 32 rows in shared memory: lane l copies row l's constants
//     (A_i, B_i, P_i, the stencil quotients, K_T(i,i), u1 and u2 at p_i) one slab ahead;
//   - streams every group's tiles through the same two-slot bulk-copy ring as k_tick_ring, the
//     copying side running on into the next slab, never beyond it.
// The tile arithmetic, the warp totals and the stores of a group are those of k_tick_ring.
// Slabs in an FP64 phase take the global-memory path of tick_group, group by group.
constexpr int kSlabWarps = 11;   // 11 warps x 2 slots x 8.5 KB + queues fit the 227 KB of an SM
constexpr int kSlabRc = 8;       // row constants per row (see above)
constexpr int kSlabRing = 4;     // records and ids: slabs k .. k + 3
struct SlabQueue {
    SlabRec rec[kSlabRing];
    int phase[kSlabRing];
    int id[kSlabRing];
    float rc[2][kSlabRc][32];    // row constants of slabs k and k + 1 (by parity), [constant][row]
};
static_assert(sizeof(SlabQueue) % 16 == 0, "slab queues must stay 16-byte aligned");
constexpr size_t kSlabTileBytes = (size_t)kSlabWarps * 2 * kTileFloats * sizeof(float);
constexpr size_t kSlabBarBytes = (size_t)kSlabWarps * 2 * 8;
constexpr size_t kSlabSmem = kSlabTileBytes + kSlabBarBytes + kSlabWarps * sizeof(SlabQueue);
static_assert(kSlabSmem <= 227 * 1024, "slab sweep shared memory");
static_assert(kSlabBarBytes % 16 == 0, "slab queues must start 16-byte aligned");
static_assert(kRows * kSlabGroups == 32, "a slab's rows are one per lane");

__global__ void __launch_bounds__(kSlabWarps * 32, 1)
    k_tick_slab(const DevInst* __restrict__ inst, const Ctl* __restrict__ ctl, Grid g, Work w,
                const float* __restrict__ Khi, const float* __restrict__ Klo, const double* A,
                const double* B, int ntot, int list, int* err) {
    constexpr int S = 2;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* ring = reinterpret_cast<float*>(smem) + (size_t)warp * S * kTileFloats;
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(smem + kSlabTileBytes) + warp * S;
    SlabQueue& q = reinterpret_cast<SlabQueue*>(smem + kSlabTileBytes + kSlabBarBytes)[warp];
    if (lane == 0) {
        for (int k = 0; k < S; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[k]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // Every warp of the grid claims slabs from one counter of the active list (the counter of the
    // next tick is cleared here); each claim is issued one slab before its result is used, so the
    // atomic's round trip overlaps a slab's work.
    if (blockIdx.x == 0 && threadIdx.x == 0) w.claim[(list + 1) % 3] = 0;
    const int nact = w.lcount[6 + list];
    const int* ids = w.slist + (size_t)list * w.n_slabs;
    int* ctr_claim = w.claim + list;
    int pending = (lane == 0) ? atomicAdd(ctr_claim, 1) : 0;
    auto claim = [&]() -> int {
        const int c = __shfl_sync(0xffffffffu, pending, 0);
        if (lane == 0) pending = (c < nact) ? atomicAdd(ctr_claim, 1) : c;
        return c < nact ? c : -1;
    };
    if (*reinterpret_cast<volatile const int*>(err)) return;
    const bool bc = (ctl->vertex == QDSE_VERTEX_BC);
    const int stall = ctl->stall_copies ? 16 : 0;
    const uint64_t pol = lane == 0 ? evict_first_policy() : evict_last_policy();

    int nmine = 1 << 30;  // slabs this warp claimed: known once a claim fails
    // the record (eight 16-byte words) and phase of slab k, whose id is in the queue
    auto request_rec = [&](int k) {
        const int id = q.id[k % kSlabRing];
        if (lane < 8) {
            cp16(reinterpret_cast<int4*>(&q.rec[k % kSlabRing]) + lane,
                 reinterpret_cast<const int4*>(g.slabs + id) + lane);
        } else if (lane == 8) {
            cp4(&q.phase[k % kSlabRing], w.sphase + id);
        }
    };
    // the row constants of slab k (record in the queue): lane l copies row 4 g0 + l's
    auto request_rc = [&](int k) {
        const SlabRec& R = q.rec[k % kSlabRing];
        const int i = kRows * R.g0 + lane;
        if (lane < kRows * R.ng && i < R.n) {
            const int o = R.x_off + i;
            float(*rc)[32] = q.rc[k & 1];
            cp4(&rc[0][lane], w.x32 + o);
            cp4(&rc[1][lane], w.x32 + ntot + o);
            cp4(&rc[2][lane], g.sp32 + o);
            cp4(&rc[3][lane], w.dia32 + o);
            cp4(&rc[4][lane], w.dia32 + ntot + o);
            cp4(&rc[5][lane], g.ktd + o);
            cp4(&rc[6][lane], w.vec32 + vpos(R.v_off + i, 2));
            cp4(&rc[7][lane], w.vec32 + vpos(R.v_off + i, 3));
        }
    };
    // prologue: ids of slabs 0 .. 2, then the records of slabs 0 and 1, then slab 0's rows
    for (int k = 0; k < 3 && k < nmine; ++k) {
        const int c = claim();
        if (c < 0) nmine = k;
        else if (lane == 0) cp4(&q.id[k], ids + c);
    }
    if (nmine == 0) return;
    cp_commit();
    cp_wait(0);
    __syncwarp();
    for (int k = 0; k < 2 && k < nmine; ++k) request_rec(k);
    cp_commit();
    cp_wait(0);
    __syncwarp();
    request_rc(0);
    cp_commit();

    // copying side: slab ps, group pg of it, its tiles from column pc while ptiles
    int ps = 0, pg = -1, pc = 0, pjhi = 0, pnr = 0, pvoff = 0;
    long long pkbase = 0;
    bool ptiles = false;
    unsigned issued = 0, consumed = 0;
    // one step of the copying side: issue one tile, or move onto the next group with tiles
    // (possibly in the next slab, never beyond the slab after the computing side's ck)
    auto produce = [&](int ck) -> bool {
        while (!ptiles) {
            int s_ = ps, g_ = pg + 1;
            if (s_ >= nmine || s_ > ck + 1) return false;
            const SlabRec* R = &q.rec[s_ % kSlabRing];
            int ph = q.phase[s_ % kSlabRing];
            if (g_ >= R->ng || (ph != PH_PICARD32 && ph != PH_TANGENT32)) {
                s_ += 1;
                g_ = 0;
                if (s_ >= nmine || s_ > ck + 1) return false;
                R = &q.rec[s_ % kSlabRing];
                ph = q.phase[s_ % kSlabRing];
                if (ph != PH_PICARD32 && ph != PH_TANGENT32) {  // an FP64 slab: no tiles
                    ps = s_;
                    pg = R->ng;
                    continue;
                }
            }
            ps = s_;
            pg = g_;
            const int2 bd = R->band[g_];
            const int i0 = kRows * (R->g0 + g_);
            if (bd.y > bd.x) {
                pc = bd.x;
                pjhi = bd.y;
                pnr = min(kRows, R->n - i0);
                pvoff = R->v_off;
                pkbase = R->k_off + 3LL * i0 * R->ld;
                ptiles = true;
            }
        }
        const int slot = issued % S;
        const uint32_t bar = smem_addr(&bars[slot]);
        const int cols = min(kTileCols, pjhi - pc);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"((uint32_t)(cols * (3 * pnr + 5) * 4 + stall))
                         : "memory");
        __syncwarp();
        if (lane < 2) {
            float* dst = ring + slot * kTileFloats + (lane ? kVecOff : 0);
            const float* src = lane ? w.vec32 + vpos(pvoff + pc, 0)
                                    : Khi + pkbase + (long long)(pc >> 2) * 3 * pnr * 4;
            bulk_copy_hint(dst, src, cols * (lane ? 5 : 3 * pnr) * 4, bar, pol);
        }
        ++issued;
        pc += kTileCols;
        if (pc >= pjhi) ptiles = false;
        return true;
    };
    auto fill = [&](int ck) {
        while (issued - consumed < (unsigned)S && produce(ck)) {
        }
    };

    const int qv = group_total_index(lane), rr = qv % kRows;
    const bool isB = qv >= kRows;
    bool ok = true;
    for (int ck = 0; ck < nmine && ok; ++ck) {
        // slab ck's rows, slab ck + 1's record and slab ck + 2's id have arrived (requested one
        // slab earlier); request slab ck + 1's rows, slab ck + 2's record, slab ck + 3's id
        cp_wait(0);
        __syncwarp();
        if (ck + 1 < nmine) request_rc(ck + 1);
        if (ck + 2 < nmine) request_rec(ck + 2);
        if (ck + 3 < nmine) {
            const int c = claim();
            if (c < 0) nmine = ck + 3;
            else if (lane == 0) cp4(&q.id[(ck + 3) % kSlabRing], ids + c);
        }
        cp_commit();
        const SlabRec& R = q.rec[ck % kSlabRing];
        const int phase = q.phase[ck % kSlabRing];
        if (phase != PH_PICARD32 && phase != PH_TANGENT32) {
            if (phase == PH_RESID64 || phase == PH_PICARD64) {
                const DevInst I = inst[R.b];
                for (int gi = 0; gi < R.ng; ++gi) {
                    GroupDesc d{};
                    d.b = R.b;
                    d.i0 = kRows * (R.g0 + gi);
                    d.nr = min(kRows, R.n - d.i0);
                    tick_group(d, phase, lane, I, ctl, g, w, Khi, Klo, A, B, ntot);
                }
            }
            continue;
        }
        const float(*rc)[32] = q.rc[ck & 1];
        const bool tan = (phase == PH_TANGENT32);
        const int collocated = (R.mode == QDSE_COLLOCATED) && bc;
        for (int gi = 0; gi < R.ng; ++gi) {
            const int i0 = kRows * (R.g0 + gi), nr = min(kRows, R.n - i0), o = R.x_off + i0;
            const int jlo = R.band[gi].x, jhi = R.band[gi].y;
            const bool full = !tan && bc && nr == kRows;
            Rows32 Rw;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                Rw.sA[r] = 0.f;
                Rw.sB[r] = 0.f;
                const bool v = r < nr;
                Rw.Ai[r] = rc[0][kRows * gi + r];
                Rw.Bi[r] = rc[1][kRows * gi + r];
                Rw.Pi[r] = rc[2][kRows * gi + r];
                Rw.dAi[r] = (tan && v) ? __ldg(w.d32 + o + r) : 0.f;
                Rw.dBi[r] = (tan && v) ? __ldg(w.d32 + ntot + o + r) : 0.f;
            }
            fill(ck);
            for (int c = jlo; c < jhi; c += kTileCols) {
                const int slot = consumed % S;
                const bool got = ring_wait(smem_addr(&bars[slot]), (consumed / S) & 1);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                const int col = c + 4 * lane;
                const int wc = min(kTileCols, jhi - c);
                const float* sl = ring + slot * kTileFloats;
                if (full && wc <= kTileCols / 4) {
                    narrow_tile32<4>(Rw, sl, c, jhi, lane);
                } else if (full && wc <= kTileCols / 2) {
                    narrow_tile32<2>(Rw, sl, c, jhi, lane);
                } else if (col < jhi) {
                    const float* vb = sl + kVecOff + lane * 20;
                    auto V4 = [&](int comp) {
                        return *reinterpret_cast<const float4*>(vb + 4 * comp);
                    };
                    const float4 a = V4(0), b = V4(1), u1 = V4(2), u2 = V4(3), u3 = V4(4);
                    if (full) {
                        const float* kb = sl + lane * (3 * kRows * 4);
                        const int sw = ((col >> 2) >> 1) & 3;
                        auto K = [&](int r, int pl) {
                            return *reinterpret_cast<const float4*>(kb + ((3 * r + pl) ^ sw) * 4);
                        };
                        rows32_chunk<false>(Rw, K, kRows, 0, true, 0, a, b, u1, u2, u3, a, a, a, a,
                                            a);
                    } else {
                        const float* kb = sl + lane * 3 * nr * 4;
                        const int sw = kswz(nr, col >> 2);
                        auto K = [&](int r, int pl) {
                            return *reinterpret_cast<const float4*>(kb + ((3 * r + pl) ^ sw) * 4);
                        };
                        if (tan) {
                            const float* db_ = w.dvec32 + vpos(R.v_off + col, 0);
                            const float4 ea = ld4(db_), eb = ld4(db_ + 4), e1 = ld4(db_ + 8),
                                         e2 = ld4(db_ + 12), e3 = ld4(db_ + 16);
                            rows32_chunk<true>(Rw, K, nr, 0, bc, 0, a, b, u1, u2, u3, ea, eb, e1,
                                               e2, e3);
                        } else {
                            rows32_chunk<false>(Rw, K, nr, 0, bc, 0, a, b, u1, u2, u3, a, a, a, a,
                                                a);
                        }
                    }
                }
                __syncwarp();
                ++consumed;
                fill(ck);
            }
            if (!ok) break;
            float tot = group_totals(Rw.sA, Rw.sB, lane);
            if (group_total_leader(lane) && rr < nr) {
                const int row = kRows * gi + rr;
                const float Pl = rc[2][row];
                if (collocated) {
                    // removable limit q^2 -> p^2 of row i0 + rr
                    const float KTd = rc[5][row], qA = rc[3][row], qB = rc[4][row];
                    const float x1 = rc[6][row], x2 = rc[7][row];
                    if (!tan) {
                        tot += isB ? (x1 * qA - x2 * qB) * KTd : (-x1 * qB - Pl * x2 * qA) * KTd;
                    } else {
                        const int ir = R.v_off + i0 + rr;
                        const float y1 = __ldg(w.dvec32 + vpos(ir, 2)),
                                    y2 = __ldg(w.dvec32 + vpos(ir, 3));
                        const float eqA = __ldg(w.ddia32 + o + rr),
                                    eqB = __ldg(w.ddia32 + ntot + o + rr);
                        tot += isB ? (y1 * qA + x1 * eqA - y2 * qB - x2 * eqB) * KTd
                                   : (-y1 * qB - x1 * eqB - Pl * (y2 * qA + x2 * eqA)) * KTd;
                    }
                }
                const float sc = R.sc32;
                if (!isB) w.xn32[o + rr] = tan ? __fdividef(sc * tot, Pl) : 1.f + __fdividef(sc * tot, Pl);
                else w.xn32[ntot + o + rr] = tan ? sc * tot : R.m32 + sc * tot;
            }
        }
    }
    cp_wait(0);  // no small copy may land after the block has released its shared memory
    if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        for (unsigned u = consumed; u < issued; ++u)
            ring_wait(smem_addr(&bars[u % S]), (u / S) & 1);
    }
}

// Advance every instance on the current active list after a tick's sweep (one block per instance,
// blocks persistent over the list).
__global__ void __launch_bounds__(kUpdThreads, 6) k_update(const DevInst* __restrict__ inst, DevState* state,
                                                const Ctl* __restrict__ ctl, Grid g, Work w,
                                                double* A, double* B, int ntot, int* count,
                                                unsigned long long* ctr, int list,
                                                const int* err) {
    // a bounded wait of this tick's sweep ran out: its outputs are incomplete, the solve stops
    if (*reinterpret_cast<volatile const int*>(err)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int clr = (list + 2) % 3;  // lists of two ticks ahead start empty
        w.lcount[clr] = 0;
        w.lcount[3 + clr] = 0;
        w.lcount[6 + clr] = 0;
        w.lcount[9 + clr] = 0;
    }
    __shared__ double sh[32];
    __shared__ float snew[2 * kMaxN];
    const BlockTeam T{sh};  // one block per instance
    const int n = w.lcount[list];
    const int* ids = w.ilist + (size_t)list * w.n_inst;
    for (int k = blockIdx.x; k < n; k += gridDim.x)
        update_instance(T, ids[k], inst, state, ctl, g, w, A, B, ntot, count, ctr,
                        (list + 1) % 3, blockDim.x == kUpdThreads ? snew : nullptr);
}

// Copy the final iterate out of the FP32 store where needed and report per-instance results.
__global__ void k_finish(const DevInst* __restrict__ inst, const DevState* __restrict__ state,
                         Work w, double* A, double* B, int ntot, double* change_out, int* iters,
                         int* status, int timed_out) {
    const int b = blockIdx.x;
    const DevInst I = inst[b];
    const DevState s = state[b];
    if (s.loc == 1) {
        for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
            A[I.x_off + j] = (double)w.x32[I.x_off + j];
            B[I.x_off + j] = (double)w.x32[ntot + I.x_off + j];
        }
    }
    if (threadIdx.x == 0) {
        if (change_out) change_out[b] = s.change;
        if (iters) iters[b] = s.iters;
        if (status) {
            int st = s.status;
            if (timed_out && s.phase != PH_DONE) st = QDSE_ERR_TIMEOUT;
            status[b] = st;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// stand-alone FP64 evaluations (residual, Jacobian-vector product)
// ------------------------------------------------------------------------------------------------
__global__ void k_prep64(const DevInst* __restrict__ inst, Grid g, Work w, const double* A,
                         const double* B, const double* vA, const double* vB, int ntot) {
    const DevInst I = inst[blockIdx.x];
    prepare_vectors<double, double>(I, g, ntot, A, B, w.vec64, ntot, I.x_off, w.dia64);
    if (vA)
        prepare_tangent<double, double, double>(I, g, ntot, A, B, vA, vB, w.dvec64, ntot, I.x_off,
                                                w.ddia64);
}

// F(x) (homogeneous = 0) or F(x) - x0 (homogeneous = 1) on the double-float kernels.
__global__ void __launch_bounds__(256) k_row_map64(const DevInst* __restrict__ inst,
                                                   const Ctl* __restrict__ ctl, Grid g, Work w,
                                                   const float* __restrict__ Khi,
                                                   const float* __restrict__ Klo,
                                                   const double* A, const double* B, double* FA,
                                                   double* FB, int ntot, int homogeneous) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= ntot) return;
    const DevInst I = inst[g.row_inst[r]];
    const int i = r - I.x_off;
    double sA, sB;
    const int2 bd = g.band[r];
    row_map<double, true>(lane, I, i, g.sp[r], A[r], B[r], w.vec64, w.dia64, ntot, Khi, Klo,
                          ctl->vertex, bd.x, bd.y, sA, sB);
    if (lane == 0) {
        const double scale = ctl->kappa * I.D;
        FA[r] = (homogeneous ? 0.0 : 1.0) + scale * sA / g.sp[r];
        FB[r] = (homogeneous ? 0.0 : I.m) + scale * sB;
    }
}

__global__ void __launch_bounds__(256) k_row_jvp64(const DevInst* __restrict__ inst,
                                                   const Ctl* __restrict__ ctl, Grid g, Work w,
                                                   const float* __restrict__ Khi,
                                                   const float* __restrict__ Klo,
                                                   const double* A, const double* B,
                                                   const double* vA, const double* vB,
                                                   double* JA, double* JB, int ntot) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= ntot) return;
    const DevInst I = inst[g.row_inst[r]];
    const int i = r - I.x_off;
    double sA, sB;
    const int2 bd = g.band[r];
    row_tangent<double, true>(lane, I, i, g.sp[r], A[r], B[r], vA[r], vB[r], w.vec64, w.dia64,
                              w.dvec64, w.ddia64, ntot, Khi, Klo, ctl->vertex, bd.x, bd.y, sA,
                              sB);
    if (lane == 0) {
        const double scale = ctl->kappa * I.D;
        JA[r] = scale * sA / g.sp[r];
        JB[r] = scale * sB;
    }
}

// R7 relative change between F and x per instance.
__global__ void k_rel64(const DevInst* __restrict__ inst, const double* A, const double* B,
                        const double* FA, const double* FB, double* rel) {
    __shared__ double sh[32];
    const DevInst I = inst[blockIdx.x];
    double bmax = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) bmax = fmax(bmax, fabs(FB[I.x_off + j]));
    bmax = block_max(bmax, sh);
    double ch = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        const int gj = I.x_off + j;
        ch = fmax(ch, fmax(rel_change(FA[gj] - A[gj], FA[gj], 0.0),
                           rel_change(FB[gj] - B[gj], FB[gj], 1e-12 * bmax)));
    }
    ch = block_max(ch, sh);
    if (threadIdx.x == 0) rel[blockIdx.x] = ch;
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
static inline int row_blocks(int ntot) { return (ntot + 7) / 8; }

cudaError_t launch_init_state(qdse_ctx* c, const Ctl& ctl, double* A, double* B, int phase0) {
    cudaError_t e = cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->work.lcount, 0, 12 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->work.claim, 0, 3 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    c->tick = 0;
    prof_begin(c, PK_OTHER);
    k_init_state<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->d_ctl, c->grid,
                                                   c->work, A, B, c->n_total, phase0);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_group_bands(qdse_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->grid.nfirst, 0, sizeof(int) * c->n_inst, c->stream);
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_OTHER);
    k_group_bands<<<(c->n_groups + 255) / 256, 256, 0, c->stream>>>(c->d_inst, c->grid,
                                                                     c->n_groups);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_group_params(qdse_ctx* c) {
    if (c->n_groups <= 0) return cudaSuccess;
    k_group_params<<<(c->n_groups + 255) / 256, 256, 0, c->stream>>>(
        c->d_inst, c->grid, c->n_groups, c->n_slabs, c->opt.cf / (8.0 * kPi * kPi * kPi));
    c->launches++;
    return cudaGetLastError();
}

template <typename Cfg>
static cudaError_t configure_ring_shape() {
    return cudaFuncSetAttribute(k_tick_ring<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg::kSmem);
}

cudaError_t configure_tick_ring() {
    cudaError_t e = configure_ring_shape<RingSweep>();
    if (e == cudaSuccess) e = configure_ring_shape<RingDeep>();
    if (e == cudaSuccess) e = configure_ring_shape<RingDeeper>();
    return e;
}

template <typename Cfg>
static void launch_ring_shape(qdse_ctx* c, double* A, double* B) {
    const int sms = c->n_sms > 0 ? c->n_sms : 152;
    const int blocks = std::max(1, std::min((c->n_groups + Cfg::kWarps - 1) / Cfg::kWarps, sms));
    k_tick_ring<Cfg><<<blocks, Cfg::kWarps * 32, Cfg::kSmem, c->stream>>>(
        c->d_inst, c->d_state, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, A, B, c->n_total,
        (int)(c->tick % 3), c->d_count, c->d_sweeps, c->fused_update, c->d_err);
}

cudaError_t launch_tick_ring(qdse_ctx* c, double* A, double* B) {
    prof_begin(c, PK_SWEEP);
    if (c->ring_shape == 1) launch_ring_shape<RingDeep>(c, A, B);
    else if (c->ring_shape == 2) launch_ring_shape<RingDeeper>(c, A, B);
    else launch_ring_shape<RingSweep>(c, A, B);
    if (c->fused_update) c->tick++;  // otherwise launch_update advances the tick
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_tick_narrow(qdse_ctx* c) {
    prof_begin(c, PK_SWEEP);
    const int sms = c->n_sms > 0 ? c->n_sms : 152;
    const int blocks = std::max(1, std::min((c->n_groups + 31) / 32, 8 * sms));
    k_tick_narrow<<<blocks, 256, 0, c->stream>>>(c->grid, c->work, c->d_Khi, c->n_total,
                                                 (int)(c->tick % 3), c->d_err);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t configure_tick_slab() {
    return cudaFuncSetAttribute(k_tick_slab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSlabSmem);
}

cudaError_t launch_tick_slab(qdse_ctx* c, double* A, double* B) {
    prof_begin(c, PK_SWEEP);
    const int sms = c->n_sms > 0 ? c->n_sms : 152;
    const int blocks = std::max(1, std::min((c->n_slabs + kSlabWarps - 1) / kSlabWarps, sms));
    k_tick_slab<<<blocks, kSlabWarps * 32, kSlabSmem, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, A, B, c->n_total,
        (int)(c->tick % 3), c->d_err);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_tick(qdse_ctx* c, double* A, double* B) {
    prof_begin(c, PK_SWEEP);
    const int blocks =
        std::min((c->n_groups + 7) / 8, kTickBlocksPerSM * (c->n_sms > 0 ? c->n_sms : 152));
    k_tick<<<blocks, 256, 0, c->stream>>>(c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi,
                                          c->d_Klo, A, B, c->n_total, (int)(c->tick % 3));
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_update(qdse_ctx* c, double* A, double* B) {
    prof_begin(c, PK_UPDATE);
    const int blocks = std::min(c->n_inst, 16 * (c->n_sms > 0 ? c->n_sms : 152));
    k_update<<<blocks, 128, 0, c->stream>>>(c->d_inst, c->d_state, c->d_ctl, c->grid, c->work,
                                            A, B, c->n_total, c->d_count, c->d_sweeps,
                                            (int)(c->tick % 3), c->d_err);
    c->tick++;
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_sweep_otf(qdse_ctx* c, const double* A, const double* B, double* FA,
                             double* FB, int only_active) {
    prof_begin(c, PK_SWEEP);
    const int blocks = (c->n_total + kOtfRowsPerBlock - 1) / kOtfRowsPerBlock;
    k_sweep_otf<<<blocks, 32 * kOtfRowsPerBlock, 0, c->stream>>>(
        c->d_inst, c->d_state, c->d_ctl, c->grid, c->work, A, B, FA, FB, c->n_total, only_active);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_finish(qdse_ctx* c, double* A, double* B, double* change_out, int* iters,
                          int* status) {
    prof_begin(c, PK_OTHER);
    k_finish<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->work, A, B, c->n_total,
                                               change_out, iters, status, 0);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_finish_timeout(qdse_ctx* c, double* A, double* B, double* change_out,
                                  int* iters, int* status) {
    prof_begin(c, PK_OTHER);
    k_finish<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->work, A, B, c->n_total,
                                               change_out, iters, status, 1);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_prep64(qdse_ctx* c, const double* A, const double* B, const double* vA,
                          const double* vB) {
    prof_begin(c, PK_OTHER);
    k_prep64<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, c->grid, c->work, A, B, vA, vB,
                                               c->n_total);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_residual_fp64(qdse_ctx* c, const double* A, const double* B, double* FA,
                                 double* FB, double* rel, int homogeneous, const float* Khi,
                                 const float* Klo) {
    cudaError_t e = launch_prep64(c, A, B, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_SWEEP);
    k_row_map64<<<row_blocks(c->n_total), 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, Khi, Klo, A, B, FA, FB, c->n_total, homogeneous);
    c->launches++;
    prof_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess || !rel) return e;
    prof_begin(c, PK_OTHER);
    k_rel64<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, A, B, FA, FB, rel);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_jvp(qdse_ctx* c, const double* A, const double* B, const double* vA,
                       const double* vB, double* JA, double* JB) {
    cudaError_t e = launch_prep64(c, A, B, vA, vB);
    if (e != cudaSuccess) return e;
    prof_begin(c, PK_SWEEP);
    k_row_jvp64<<<row_blocks(c->n_total), 256, 0, c->stream>>>(
        c->d_inst, c->d_ctl, c->grid, c->work, c->d_Khi, c->d_Klo, A, B, vA, vB, JA, JB,
        c->n_total);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t launch_rel64(qdse_ctx* c, const double* A, const double* B, const double* FA,
                         const double* FB, double* rel) {
    prof_begin(c, PK_OTHER);
    k_rel64<<<c->n_inst, 256, 0, c->stream>>>(c->d_inst, A, B, FA, FB, rel);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

}  // namespace qdse
