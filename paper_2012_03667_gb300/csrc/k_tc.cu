// k_tc.cu -- the FP32 Picard sweep of a batch whose instances share one kernel matrix (same grid
// and omega: a scan of m or D), as a product on the tensor cores.
//
// The BC sweep of row i of instance b (the pair terms of k_sweep.cu: pair32) is linear in the
// kernel planes K_0, K^_T = K_T/(Q - P), K_3 once the pair's row and column factors are
// separated.  With a, b, u1, u2, u3 the node vectors of instance b at q_j and h1 = 3/2 u1,
// h2 = 1/2 u2, h3 = 1/2 u3:
//   S_A(i) = -P_i G0 + P_i A_i G1 - G2 + A_i G3 + B_i G4 + A_i G7 + G8
//   S_B(i) =  G5 - A_i G4 + B_i G6 + A_i G9 + G10
// where G_f(i) = sum_j K_plane(f)(i, j) v_f(j) for the eleven column functions
//   K^_T: v0 = h2 a, v1 = h2, v2 = h3 a + u1 b, v3 = h3, v4 = u1, v5 = u1 a - u2 b, v6 = u2
//   K_3:  v7 = h2, v8 = h2 a          K_0: v9 = h1, v10 = h1 a
// (the sums of Eqs. A-B of the BC equation with the pair factors expanded).  For the whole batch
// this is the product G = V K^T of the column functions V [(function, instance) x N] and the
// plane of each function, [N x N], which runs as tcgen05 MMAs with FP32 accumulation in tensor
// memory: M = 128 (function, instance) rows, N = 256 kernel rows i, K = the columns j.  The
// operands are split into TF32 parts, x = hi + lo, and each product is hi*hi + hi*lo + lo*hi
// ("3xTF32": the dropped lo*lo term is below 2^-21 of the product), i.e. one TF32 product over
// three times the K extent with the operands [V_hi | V_hi | V_lo] and [K_hi | K_lo | K_hi].
//
// Expanding the differences (a_j - A_i) cancels where K^_T ~ 1/(Q - P) is large, i.e. near the
// diagonal (the cancellation factor falls like 1/|i - j|).  So the product uses the far field only
// (|i - j| > kTcW, the band set to zero) and the near band |i - j| <= kTcW is summed in the
// difference form, in FP32 on the CUDA cores, by the combining kernel (k_tc_combine), which also
// adds the collocated removable-limit term as in the ring sweep and forms the new A_i, B_i.
//
// The product kernel (k_tc_gemm): one CTA per 128 (function, instance) rows x 256 kernel rows;
// 4 warps.  Thread 0 streams the operand tiles by tensor-map copies through a 4-stage shared-memory
// ring, thread 32 issues the MMAs (M = 128, N = 256, K = 8), then all 128 threads read their row
// of the accumulator and store it.  Every wait is bounded: on expiry the kernel sets the error flag,
// skips the rest, frees its tensor memory and returns.
#include <cuda.h>

#include <cstdio>

#include "qdse_internal.h"
#include "tc_sm100.cuh"

namespace qdse {

constexpr int kTcM = 128;     // (function, instance) rows per CTA
constexpr int kTcN = 256;     // kernel rows i per CTA
constexpr int kTcK = 32;      // K values per stage (one 128-byte swizzle row)
constexpr int kTcStages = 4;
constexpr int kTcF = 11;      // column functions
constexpr int kTcW = 8;       // near band: |i - j| <= kTcW in the difference form
constexpr int kTcNW = 2 * kTcW + 1;
constexpr uint32_t kTcAbytes = kTcM * kTcK * 4;                 // 16 KB
constexpr uint32_t kTcBbytes = kTcN * kTcK * 4;                 // 32 KB
constexpr uint32_t kTcStageBytes = kTcAbytes + kTcBbytes;       // 48 KB
constexpr size_t kTcSmem = kTcStages * (size_t)kTcStageBytes + 1024 + 256;
constexpr long long kTcWaitBudget = 2000000000LL;  // clock cycles (about 1 s)
static_assert(kTcSmem <= 227 * 1024, "tensor-core product shared memory");
static_assert(kTcStageBytes % 1024 == 0 && kTcAbytes % 1024 == 0,
              "operand tiles start on 1024-byte boundaries");
// the plane of function f: 1 (K^_T) for f < 7, 2 (K_3) for 7, 8, 0 (K_0) for 9, 10
__host__ __device__ constexpr int tc_plane(int f) { return f < 7 ? 1 : (f < 9 ? 2 : 0); }

// ---- operands ------------------------------------------------------------------------------
// The far-field planes (band |i - j| <= kTcW zeroed; entries outside the row's stored band are
// zero) as TF32 parts and the near band, from the pool block of instance 0.  Kf: [2][3 N][ldk]
// row-major, the high parts then the low parts.  The batch shares that block, so the precompute
// ran for instance 0 only: its K_T(i, i) (the removable-limit factor) is copied to every instance.
__global__ void k_tc_extract(const DevInst* __restrict__ inst, Grid g, const float* __restrict__ Khi,
                             float* __restrict__ Kf, float* __restrict__ Kn, int ldk, int n_inst) {
    const DevInst I = inst[0];
    const int n = I.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n_inst * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), i = (int)(e % n);
        if (b > 0) g.ktd[inst[b].x_off + i] = g.ktd[I.x_off + i];
    }
    const long long total = 3LL * n * ldk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ldk);
        const int row = (int)(e / ldk);
        const int p = row / n, i = row % n;
        const int2 bd = g.band[I.x_off + i];
        float v = 0.f;
        if (j < n && j >= bd.x && j < bd.y) v = Khi[kpos(I.k_off, n, I.ld, i, p, j)];
        const int d = j - i;
        float hi = 0.f, lo = 0.f;
        if (d >= -kTcW && d <= kTcW) {
            if (j < n) Kn[((size_t)p * n + i) * kTcNW + d + kTcW] = v;
        } else {
            hi = tc::to_tf32(v);
            lo = tc::to_tf32(v - hi);
        }
        Kf[e] = hi;
        Kf[total + e] = lo;
    }
    // near-band slots outside [0, n)
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3LL * n * kTcNW;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e % kTcNW), i = (int)((e / kTcNW) % n);
        const int j = i + t - kTcW;
        if (j < 0 || j >= n) Kn[e] = 0.f;
    }
}

// The column functions of every instance as TF32 parts: V[part][f * bp + b][j] (part 0 high, 1 low;
// bp = the batch padded to a multiple of 128, so that a 128-row tile holds one function; ldv
// columns; zero beyond n, for b >= n_inst and for instances outside the FP32 Picard phase).
__global__ void k_tc_prep(const DevInst* __restrict__ inst, const DevState* __restrict__ state,
                          Work w, float* __restrict__ V, int n, int n_inst, int bp, int ldv) {
    const long long total = (long long)bp * ldv;
    const size_t part = (size_t)kTcF * bp * ldv;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ldv), b = (int)(e / ldv);
        float f[kTcF];
#pragma unroll
        for (int k = 0; k < kTcF; ++k) f[k] = 0.f;
        if (b < n_inst && j < n && state[b].phase == PH_PICARD32) {
            const int x = inst[b].v_off + j;
            const float a = w.vec32[vpos(x, 0)], bb = w.vec32[vpos(x, 1)];
            const float u1 = w.vec32[vpos(x, 2)], u2 = w.vec32[vpos(x, 3)], u3 = w.vec32[vpos(x, 4)];
            const float h1 = 1.5f * u1, h2 = 0.5f * u2, h3 = 0.5f * u3;
            f[0] = h2 * a;
            f[1] = h2;
            f[2] = fmaf(h3, a, u1 * bb);
            f[3] = h3;
            f[4] = u1;
            f[5] = fmaf(u1, a, -u2 * bb);
            f[6] = u2;
            f[7] = h2;
            f[8] = h2 * a;
            f[9] = h1;
            f[10] = h1 * a;
        }
#pragma unroll
        for (int k = 0; k < kTcF; ++k) {
            const size_t at = ((size_t)k * bp + b) * ldv + j;
            const float hi = tc::to_tf32(f[k]);
            V[at] = hi;
            V[part + at] = tc::to_tf32(f[k] - hi);
        }
    }
}

// ---- the product ---------------------------------------------------------------------------
// G[f * bp + b][i] = sum_j V_f,b(j) K_plane(f)(i, j) for the far field, 3xTF32.
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapV, const __grid_constant__ CUtensorMap mapK,
              float* __restrict__ G, int n, int bp, int ldg, const int* __restrict__ any,
              int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // 1024-byte alignment of the stage tiles (the dynamic window's base is only 16-byte aligned)
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* tail = smem + kTcStages * (size_t)kTcStageBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty = full + kTcStages;
    uint64_t* done = empty + kTcStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_bad;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int mt = blockIdx.x, nt = blockIdx.y;
    const int r0 = mt * kTcM, i0 = nt * kTcN;
    if (*reinterpret_cast<volatile const int*>(err)) return;  // an earlier wait ran out
    // no instance of this tile's 128 rows is in the FP32 Picard phase
    if (!any[(r0 % bp) / kTcM]) return;
    const int plane = tc_plane(r0 / bp);

    if (tid == 0) s_bad = 0;
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    // steps: 32 values of K each, three per K block (hi*hi, hi*lo, lo*hi)
    const int nsteps = 3 * ((n + kTcK - 1) / kTcK);

    if (tid == 0) {
        // producer: the V tile (rows part 11 bp + r0 ..) and the K tile (rows part 3 n + plane n +
        // i0 ..)
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % kTcStages, k = t / 3, u = t % 3;
            if (t >= kTcStages &&
                !tc::mbar_wait(&empty[s], ((t / kTcStages) - 1) & 1, kTcWaitBudget)) {
                s_bad = 1;
                break;
            }
            unsigned char* st = smem + (size_t)s * kTcStageBytes;
            tc::mbar_expect_tx(&full[s], kTcStageBytes);
            tc::tma_load_2d(st, &mapV, k * kTcK, (u == 2 ? kTcF * bp : 0) + r0, &full[s]);
            tc::tma_load_2d(st + kTcAbytes, &mapK, k * kTcK, ((u == 1 ? 3 : 0) + plane) * n + i0,
                            &full[s]);
        }
    } else if (tid == 32) {
        constexpr uint32_t idesc = tc::idesc_tf32(kTcM, kTcN);
        bool ok = true;
        for (int t = 0; t < nsteps && ok; ++t) {
            const int s = t % kTcStages;
            if (!tc::mbar_wait(&full[s], (t / kTcStages) & 1, kTcWaitBudget)) {
                ok = false;
                s_bad = 1;
                break;
            }
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_u32(smem + (size_t)s * kTcStageBytes);
            const uint32_t sb = sa + kTcAbytes;
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {
                const uint32_t off = kk * 32;  // bytes along K inside the swizzled row
                tc::mma_tf32(tmem, tc::sw128_desc(sa + off), tc::sw128_desc(sb + off), idesc,
                             (t > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (ok) tc::mma_commit(done);
    }
    __syncwarp();
    const bool have = tc::mbar_wait(done, 0, kTcWaitBudget);
    tc::fence_after_sync();
    __syncthreads();
    if (!have || s_bad) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        // thread = accumulator row r0 + tid; its 256 columns are kernel rows i0 ..
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float* dst = G + (size_t)(r0 + tid) * ldg + i0;
        const int ncol = min(kTcN, n - i0);
        for (int c = 0; c < kTcN; c += 8) {
            float v[8];
            tc::tmem_ld8(trow + c, v);
            if (c + 8 <= ncol) {
                *reinterpret_cast<float4*>(dst + c) = make_float4(v[0], v[1], v[2], v[3]);
                *reinterpret_cast<float4*>(dst + c + 4) = make_float4(v[4], v[5], v[6], v[7]);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (c + q < ncol) dst[c + q] = v[q];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ---- the sweep -----------------------------------------------------------------------------
__device__ __forceinline__ void pair_near(float a, float b, float u1, float u2, float u3, float K0,
                                          float KT, float K3, float Ai, float Bi, float Pi,
                                          float& sA, float& sB) {
    // the difference form of the ring sweep's pair (h1 = 3/2 u1, h2 = 1/2 u2, h3 = 1/2 u3)
    const float h1 = 1.5f * u1, h2 = 0.5f * u2, h3 = 0.5f * u3;
    const float da = a - Ai, db = b - Bi, sa = Ai + a;
    const float T = fmaf(Pi, h2, h3);
    const float cT = fmaf(-T, da, -u1 * db);
    sA = fmaf(cT, KT, fmaf(h2 * sa, K3, sA));
    sB = fmaf(fmaf(u1, da, -u2 * db), KT, fmaf(h1 * sa, K0, sB));
}

constexpr int kCbRows = 128;  // rows i per combining block
constexpr int kCbInst = 8;    // instances per combining block

// The new A_i, B_i of every instance in the FP32 Picard phase: the far field from G, the near band
// in the difference form, the removable-limit term.  Block: 128 rows x 8 instances.
__global__ void __launch_bounds__(kCbRows) k_tc_combine(const DevInst* __restrict__ inst,
                                                        const DevState* __restrict__ state,
                                                        const GroupDesc* __restrict__ gdesc,
                                                        Grid g, Work w, const float* __restrict__ G,
                                                        const float* __restrict__ Kn, int n,
                                                        int n_inst, int bp, int ldg, int ntot) {
    constexpr int NV = kCbRows + 2 * kTcW;
    __shared__ float sV[kCbInst][5][NV];
    __shared__ int s_ph[kCbInst], s_x[kCbInst], s_v[kCbInst];
    __shared__ float s_sc[kCbInst], s_m[kCbInst];
    const int m0 = blockIdx.x * kCbRows, b0 = blockIdx.y * kCbInst, r = threadIdx.x;
    if (r < kCbInst) {
        const int b = b0 + r;
        int ph = PH_DONE;
        if (b < n_inst) {
            const DevInst I = inst[b];
            ph = state[b].phase;
            s_x[r] = I.x_off;
            s_v[r] = I.v_off;
            const GroupDesc d = gdesc[I.g_off];
            s_sc[r] = d.sc32;
            s_m[r] = d.m32;
        }
        s_ph[r] = ph;
    }
    __syncthreads();
    for (int e = r; e < kCbInst * 5 * NV; e += kCbRows) {
        const int jj = e % NV, c = (e / NV) % 5, q = e / (5 * NV);
        const int j = m0 - kTcW + jj;
        float v = 0.f;
        if (j >= 0 && j < n && s_ph[q] == PH_PICARD32) v = w.vec32[vpos(s_v[q] + j, c)];
        sV[q][c][jj] = v;
    }
    __syncthreads();
    const int i = m0 + r;
    if (i >= n) return;
    const int x0 = inst[0].x_off;
    const float Pi = g.sp32[x0 + i], KTd = g.ktd[x0 + i];
    float kn[3][kTcNW];  // this row's near band, for every instance of the block
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int t = 0; t < kTcNW; ++t) kn[p][t] = Kn[((size_t)p * n + i) * kTcNW + t];
    for (int q = 0; q < kCbInst; ++q) {
        const int b = b0 + q;
        if (s_ph[q] != PH_PICARD32) continue;
        float Gf[kTcF];
#pragma unroll
        for (int f = 0; f < kTcF; ++f) Gf[f] = G[((size_t)f * bp + b) * ldg + i];
        const int o = s_x[q];
        const float Ai = w.x32[o + i], Bi = w.x32[ntot + o + i];
        float sA = -Pi * Gf[0] + Pi * Ai * Gf[1] - Gf[2] + Ai * Gf[3] + Bi * Gf[4] + Ai * Gf[7] +
                   Gf[8];
        float sB = Gf[5] - Ai * Gf[4] + Bi * Gf[6] + Ai * Gf[9] + Gf[10];
#pragma unroll
        for (int t = 0; t < kTcNW; ++t)
            pair_near(sV[q][0][r + t], sV[q][1][r + t], sV[q][2][r + t], sV[q][3][r + t],
                      sV[q][4][r + t], kn[0][t], kn[1][t], kn[2][t], Ai, Bi, Pi, sA, sB);
        // removable limit q^2 -> p^2 (collocated): K_T(i, i) times the stencil quotients
        const float x1 = sV[q][2][r + kTcW], x2 = sV[q][3][r + kTcW];
        const float qA = w.dia32[o + i], qB = w.dia32[ntot + o + i];
        sA += (-x1 * qB - Pi * x2 * qA) * KTd;
        sB += (x1 * qA - x2 * qB) * KTd;
        const float sc = s_sc[q];
        w.xn32[o + i] = 1.f + __fdividef(sc * sA, Pi);
        w.xn32[ntot + o + i] = s_m[q] + sc * sB;
    }
}

// Which 128-instance blocks hold an instance in the FP32 Picard phase (the product skips the
// others).
__global__ void k_tc_any(const DevState* __restrict__ state, int n_inst, int nblk, int* any) {
    const int k = blockIdx.x;
    if (k >= nblk) return;
    int f = 0;
    for (int b = k * kTcM + threadIdx.x; b < min(n_inst, (k + 1) * kTcM); b += blockDim.x)
        f |= state[b].phase == PH_PICARD32;
    f = __syncthreads_or(f);
    if (threadIdx.x == 0) any[k] = f;
}

// ---- host side ------------------------------------------------------------------------------
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// A 2-D FP32 tensor map: rows x cols (row stride ld floats), boxes of 32 columns x box_rows rows,
// 128-byte swizzle, zero fill outside.
static bool make_map(CUtensorMap* m, const float* base, long long rows, int cols, int ld,
                     int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t tc_setup(qdse_ctx* c) {
    const int n = c->tc_n;
    c->tc_ld = (n + kTcK - 1) / kTcK * kTcK;
    c->tc_bp = (c->n_inst + kTcM - 1) / kTcM * kTcM;
    c->tc_ldg = (n + 3) / 4 * 4;
    const size_t vrows = (size_t)2 * kTcF * c->tc_bp;
    cudaError_t e = cudaMalloc((void**)&c->tc_Kf, sizeof(float) * 6 * (size_t)n * c->tc_ld);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->tc_Kn, sizeof(float) * 3 * (size_t)n * kTcNW);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->tc_V, sizeof(float) * vrows * c->tc_ld);
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&c->tc_G, sizeof(float) * (size_t)kTcF * c->tc_bp * c->tc_ldg);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->tc_any, sizeof(int) * (c->tc_bp / kTcM));
    if (e != cudaSuccess) return e;
    e = cudaMemset(c->tc_V, 0, sizeof(float) * vrows * c->tc_ld);
    if (e != cudaSuccess) return e;
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    if (!make_map(reinterpret_cast<CUtensorMap*>(c->tc_map[0]), c->tc_V, (long long)vrows,
                  c->tc_ld, c->tc_ld, kTcM) ||
        !make_map(reinterpret_cast<CUtensorMap*>(c->tc_map[1]), c->tc_Kf, 6LL * n, c->tc_ld,
                  c->tc_ld, kTcN))
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTcSmem);
}

void tc_free(qdse_ctx* c) {
    for (float** p : {&c->tc_Kf, &c->tc_Kn, &c->tc_V, &c->tc_G}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    if (c->tc_any) cudaFree(c->tc_any);
    c->tc_any = nullptr;
}

cudaError_t launch_tc_extract(qdse_ctx* c) {
    const long long total = 3LL * c->tc_n * c->tc_ld;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    k_tc_extract<<<blocks, 256, 0, c->stream>>>(c->d_inst, c->grid, c->d_Khi, c->tc_Kf, c->tc_Kn,
                                                c->tc_ld, c->n_inst);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_tc_sweep(qdse_ctx* c) {
    prof_begin(c, PK_SWEEP);
    const int nblk = c->tc_bp / kTcM;
    k_tc_any<<<nblk, 128, 0, c->stream>>>(c->d_state, c->n_inst, nblk, c->tc_any);
    const long long total = (long long)c->tc_bp * c->tc_ld;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    k_tc_prep<<<blocks, 256, 0, c->stream>>>(c->d_inst, c->d_state, c->work, c->tc_V, c->tc_n,
                                             c->n_inst, c->tc_bp, c->tc_ld);
    const dim3 gg(kTcF * c->tc_bp / kTcM, (c->tc_n + kTcN - 1) / kTcN);
    k_tc_gemm<<<gg, 128, kTcSmem, c->stream>>>(
        *reinterpret_cast<const CUtensorMap*>(c->tc_map[0]),
        *reinterpret_cast<const CUtensorMap*>(c->tc_map[1]), c->tc_G, c->tc_n, c->tc_bp,
        c->tc_ldg, c->tc_any, c->d_err);
    const dim3 gc((c->tc_n + kCbRows - 1) / kCbRows, (c->n_inst + kCbInst - 1) / kCbInst);
    k_tc_combine<<<gc, kCbRows, 0, c->stream>>>(c->d_inst, c->d_state, c->grid.gdesc, c->grid,
                                               c->work, c->tc_G, c->tc_Kn, c->tc_n, c->n_inst,
                                               c->tc_bp, c->tc_ldg, c->n_total);
    c->launches += 4;
    prof_end(c);
    return cudaGetLastError();
}

}  // namespace qdse
