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
// this is three matrix products, K_plane [N x N] times [N x (functions x instances)], which run
// here as tcgen05 MMAs with FP32 accumulation in tensor memory.  The operands are split into TF32
// parts, x = hi + lo, and each product is hi*hi + hi*lo + lo*hi ("3xTF32": the dropped lo*lo term
// is below 2^-21 of the product), i.e. one TF32 product over three times the K extent with the
// operands [A_hi | A_hi | A_lo] and [B_hi | B_lo | B_hi].
//
// Expanding the differences (a_j - A_i) cancels where K^_T ~ 1/(Q - P) is large, i.e. near the
// diagonal (the cancellation factor falls like 1/|i - j|).  So the product uses the far field only
// (|i - j| > kTcW, the band set to zero) and the near band |i - j| <= kTcW is summed in the
// difference form, in FP32 on the CUDA cores, in the epilogue of the same kernel; the collocated
// removable-limit term follows as in the ring sweep.
//
// One CTA: 128 rows i x 16 instances; 4 warps.  Thread 0 streams the operand tiles by tensor-map
// copies through a 3-stage shared-memory ring, thread 32 issues the MMAs (3 per 8 values of K:
// K^_T with 7 x 16 columns, K_3 and K_0 with 2 x 16 each), then all 128 threads read their row's
// accumulators and finish the sweep of the rows of the instances that are in the FP32 Picard phase.
// Every wait is bounded: on expiry the kernel sets the error flag, skips the rest, frees its tensor
// memory and returns.
#include <cuda.h>

#include <cstdio>

#include "qdse_internal.h"
#include "tc_sm100.cuh"

namespace qdse {

constexpr int kTcM = 128;     // rows per CTA
constexpr int kTcB = 16;      // instances per CTA
constexpr int kTcK = 32;      // K values per stage (one 128-byte swizzle row)
constexpr int kTcStages = 3;
constexpr int kTcNT = 7 * kTcB, kTcN3 = 2 * kTcB, kTcN0 = 2 * kTcB;  // MMA widths
constexpr int kTcRowsB = kTcNT + kTcN3 + kTcN0;                        // 176 operand rows
constexpr int kTcC3 = 128, kTcC0 = 160;  // tensor-memory columns of the K_3 and K_0 products
                                         // (K^_T's are 0 .. 111); 256 columns allocated
constexpr int kTcW = 8;       // near band: |i - j| <= kTcW in the difference form
constexpr int kTcNW = 2 * kTcW + 1;
constexpr int kTcQ = 8;       // instances per epilogue pass
constexpr uint32_t kTcAbytes = kTcM * kTcK * 4;                 // one plane tile: 16 KB
constexpr uint32_t kTcStageBytes = 3 * kTcAbytes + kTcRowsB * kTcK * 4;  // 71680
constexpr size_t kTcSmem = kTcStages * (size_t)kTcStageBytes + 1024 + 256;
static_assert(kTcStageBytes % 1024 == 0 && (kTcNT * 128) % 1024 == 0 &&
                  ((kTcNT + kTcN3) * 128) % 1024 == 0,
              "operand tiles start on 1024-byte boundaries");
constexpr long long kTcWaitBudget = 2000000000LL;  // clock cycles (about 1 s)
static_assert(kTcSmem <= 227 * 1024, "tensor-core sweep shared memory");
static_assert(3 * kTcM * kTcNW * 4 + kTcQ * 5 * (kTcM + 2 * kTcW) * 4 <=
                  kTcStages * (size_t)kTcStageBytes,
              "the epilogue's near-band tiles fit in the freed stages");

struct TcArgs {
    const DevInst* inst;
    const DevState* state;
    const GroupDesc* gdesc;
    Grid g;
    Work w;
    const float* Kn;   // [3][N][kTcNW] near band (plane, row, j - i + kTcW)
    int n, n_inst, ntot, nbt;
    int* err;
};

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

// The column functions of every instance as TF32 parts, in the CTA-blocked layout
// V[bt][part][f * kTcB + bl][j] (bt = b / kTcB, bl = b % kTcB, part 0 high, 1 low; ldv columns, zero
// beyond n and for b >= n_inst).
__global__ void k_tc_prep(const DevInst* __restrict__ inst, Work w, float* __restrict__ V, int n,
                          int n_inst, int nbt, int ldv) {
    const long long total = (long long)nbt * kTcB * ldv;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ldv);
        const int bb = (int)(e / ldv);  // bt * 32 + bl
        const int bt = bb / kTcB, bl = bb % kTcB;
        float f[11];
#pragma unroll
        for (int k = 0; k < 11; ++k) f[k] = 0.f;
        if (bb < n_inst && j < n) {
            const int x = inst[bb].v_off + j;
            const float a = w.vec32[vpos(x, 0)], b = w.vec32[vpos(x, 1)];
            const float u1 = w.vec32[vpos(x, 2)], u2 = w.vec32[vpos(x, 3)], u3 = w.vec32[vpos(x, 4)];
            const float h1 = 1.5f * u1, h2 = 0.5f * u2, h3 = 0.5f * u3;
            f[0] = h2 * a;
            f[1] = h2;
            f[2] = fmaf(h3, a, u1 * b);
            f[3] = h3;
            f[4] = u1;
            f[5] = fmaf(u1, a, -u2 * b);
            f[6] = u2;
            f[7] = h2;
            f[8] = h2 * a;
            f[9] = h1;
            f[10] = h1 * a;
        }
        float* base = V + (size_t)bt * 2 * kTcRowsB * ldv + j;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float hi = tc::to_tf32(f[k]);
            base[(size_t)(k * kTcB + bl) * ldv] = hi;
            base[(size_t)(kTcRowsB + k * kTcB + bl) * ldv] = tc::to_tf32(f[k] - hi);
        }
    }
}

// ---- the product and the sweep -------------------------------------------------------------
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

__global__ void __launch_bounds__(128, 1)
    k_tc_sweep(const __grid_constant__ CUtensorMap mapK, const __grid_constant__ CUtensorMap mapVT,
               const __grid_constant__ CUtensorMap mapV2, TcArgs args) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // 1024-byte alignment of the stage tiles (the dynamic window's base is only 16-byte aligned)
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* tail = smem + kTcStages * (size_t)kTcStageBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty = full + kTcStages;
    uint64_t* done = empty + kTcStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_phase[kTcB], s_xoff[kTcB], s_voff[kTcB];
    __shared__ float s_sc[kTcB], s_m[kTcB];
    __shared__ int s_any, s_bad;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int mt = blockIdx.x, bt = blockIdx.y;
    const int m0 = mt * kTcM, b0 = bt * kTcB, n = args.n;
    if (*reinterpret_cast<volatile const int*>(args.err)) return;  // an earlier wait ran out

    if (tid < kTcB) {
        const int b = b0 + tid;
        int ph = PH_DONE;
        if (b < args.n_inst) {
            const DevInst I = args.inst[b];
            ph = args.state[b].phase;
            s_xoff[tid] = I.x_off;
            s_voff[tid] = I.v_off;
            const GroupDesc d = args.gdesc[I.g_off];
            s_sc[tid] = d.sc32;
            s_m[tid] = d.m32;
        }
        s_phase[tid] = ph;
    }
    if (tid == 0) {
        s_any = 0;
        s_bad = 0;
    }
    __syncthreads();
    if (tid < kTcB && s_phase[tid] == PH_PICARD32) atomicOr(&s_any, 1);
    __syncthreads();
    if (!s_any) return;  // no instance of this block is in the FP32 Picard phase

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
        // producer: the three plane tiles (rows part 3 N + p N + m0 ..) and the three
        // column-function tiles (rows bt 2 R + part R ..)
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % kTcStages, k = t / 3, u = t % 3;
            if (t >= kTcStages &&
                !tc::mbar_wait(&empty[s], ((t / kTcStages) - 1) & 1, kTcWaitBudget)) {
                s_bad = 1;
                break;
            }
            unsigned char* st = smem + (size_t)s * kTcStageBytes;
            tc::mbar_expect_tx(&full[s], kTcStageBytes);
            const int ya = (u == 2 ? 3 * n : 0) + m0;
            for (int p = 0; p < 3; ++p)
                tc::tma_load_2d(st + p * kTcAbytes, &mapK, k * kTcK, ya + p * n, &full[s]);
            unsigned char* sb = st + 3 * kTcAbytes;
            const int y = bt * 2 * kTcRowsB + (u == 1 ? kTcRowsB : 0);
            tc::tma_load_2d(sb, &mapVT, k * kTcK, y, &full[s]);
            tc::tma_load_2d(sb + kTcNT * 128, &mapV2, k * kTcK, y + kTcNT, &full[s]);
            tc::tma_load_2d(sb + (kTcNT + kTcN3) * 128, &mapV2, k * kTcK, y + kTcNT + kTcN3,
                            &full[s]);
        }
    } else if (tid == 32) {
        // MMA issuer: K^_T x (7 functions), K_3 x (2), K_0 x (2) per 8 values of K
        constexpr uint32_t iT = tc::idesc_tf32(kTcM, kTcNT), i2 = tc::idesc_tf32(kTcM, kTcN3);
        bool ok = true;
        for (int t = 0; t < nsteps && ok; ++t) {
            const int s = t % kTcStages;
            if (!tc::mbar_wait(&full[s], (t / kTcStages) & 1, kTcWaitBudget)) {
                ok = false;
                s_bad = 1;
                break;
            }
            tc::fence_after_sync();
            const uint32_t st = tc::smem_u32(smem + (size_t)s * kTcStageBytes);
            const uint32_t sb = st + 3 * kTcAbytes;
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {
                const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
                const uint32_t off = kk * 32;  // bytes along K inside the swizzled row
                tc::mma_tf32(tmem, tc::sw128_desc(st + 1 * kTcAbytes + off),
                             tc::sw128_desc(sb + off), iT, acc);
                tc::mma_tf32(tmem + kTcC3, tc::sw128_desc(st + 2 * kTcAbytes + off),
                             tc::sw128_desc(sb + kTcNT * 128 + off), i2, acc);
                tc::mma_tf32(tmem + kTcC0, tc::sw128_desc(st + off),
                             tc::sw128_desc(sb + (kTcNT + kTcN3) * 128 + off), i2, acc);
            }
            tc::mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (ok) tc::mma_commit(done);
    }
    __syncwarp();
    // every thread: the accumulators are complete
    const bool have = tc::mbar_wait(done, 0, kTcWaitBudget);
    tc::fence_after_sync();
    __syncthreads();
    if (!have || s_bad) {
        if (tid == 0) atomicExch(args.err, 1);
    } else {
        // epilogue: thread = row i, passes of kTcQ instances
        float* sKn = reinterpret_cast<float*>(smem);             // [3][kTcM][kTcNW]
        float* sV = sKn + 3 * kTcM * kTcNW;                      // [kTcQ][5][kTcM + 2 kTcW]
        constexpr int NV = kTcM + 2 * kTcW;
        for (int e = tid; e < 3 * kTcM * kTcNW; e += 128) {
            const int t = e % kTcNW, r = (e / kTcNW) % kTcM, p = e / (kTcNW * kTcM);
            const int i = m0 + r;
            sKn[e] = i < n ? args.Kn[((size_t)p * n + i) * kTcNW + t] : 0.f;
        }
        const int r = tid, i = m0 + r;
        const float Pi = i < n ? args.g.sp32[s_xoff[0] + i] : 1.f;
        const float KTd = i < n ? args.g.ktd[s_xoff[0] + i] : 0.f;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int q0 = 0; q0 < kTcB; q0 += kTcQ) {
            __syncthreads();  // the previous pass is done with sV
            for (int e = tid; e < kTcQ * 5 * NV; e += 128) {
                const int jj = e % NV, c = (e / NV) % 5, q = e / (5 * NV);
                const int j = m0 - kTcW + jj, bl = q0 + q;
                float v = 0.f;
                if (j >= 0 && j < n && s_phase[bl] == PH_PICARD32)
                    v = args.w.vec32[vpos(s_voff[bl] + j, c)];
                sV[e] = v;
            }
            __syncthreads();
            float G[11][kTcQ];
#pragma unroll
            for (int f = 0; f < 7; ++f) tc::tmem_ld8(trow + f * kTcB + q0, G[f]);
#pragma unroll
            for (int f = 0; f < 2; ++f) tc::tmem_ld8(trow + kTcC3 + f * kTcB + q0, G[7 + f]);
#pragma unroll
            for (int f = 0; f < 2; ++f) tc::tmem_ld8(trow + kTcC0 + f * kTcB + q0, G[9 + f]);
#pragma unroll
            for (int q = 0; q < kTcQ; ++q) {
                const int bl = q0 + q;
                if (i >= n || s_phase[bl] != PH_PICARD32) continue;
                const int o = s_xoff[bl];
                const float Ai = args.w.x32[o + i], Bi = args.w.x32[args.ntot + o + i];
                float sA = -Pi * G[0][q] + Pi * Ai * G[1][q] - G[2][q] + Ai * G[3][q] +
                           Bi * G[4][q] + Ai * G[7][q] + G[8][q];
                float sB = G[5][q] - Ai * G[4][q] + Bi * G[6][q] + Ai * G[9][q] + G[10][q];
                const float* v = sV + q * 5 * NV + r;  // node j = i - kTcW + t at v[c NV + t]
                const float* kn = sKn + r * kTcNW;
                for (int t = 0; t < kTcNW; ++t) {
                    pair_near(v[t], v[NV + t], v[2 * NV + t], v[3 * NV + t], v[4 * NV + t],
                              kn[t], kn[kTcM * kTcNW + t], kn[2 * kTcM * kTcNW + t], Ai, Bi, Pi,
                              sA, sB);
                }
                // removable limit q^2 -> p^2 (collocated): K_T(i, i) times the stencil quotients
                const float x1 = v[2 * NV + kTcW], x2 = v[3 * NV + kTcW];
                const float qA = args.w.dia32[o + i], qB = args.w.dia32[args.ntot + o + i];
                sA += (-x1 * qB - Pi * x2 * qA) * KTd;
                sB += (x1 * qA - x2 * qB) * KTd;
                const float sc = s_sc[bl];
                args.w.xn32[o + i] = 1.f + __fdividef(sc * sA, Pi);
                args.w.xn32[args.ntot + o + i] = s_m[bl] + sc * sB;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
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
    c->tc_nbt = (c->n_inst + kTcB - 1) / kTcB;
    const size_t vrows = (size_t)c->tc_nbt * 2 * kTcRowsB;
    cudaError_t e = cudaMalloc((void**)&c->tc_Kf, sizeof(float) * 6 * (size_t)n * c->tc_ld);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->tc_Kn, sizeof(float) * 3 * (size_t)n * kTcNW);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->tc_V, sizeof(float) * vrows * c->tc_ld);
    if (e != cudaSuccess) return e;
    e = cudaMemset(c->tc_V, 0, sizeof(float) * vrows * c->tc_ld);
    if (e != cudaSuccess) return e;
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    if (!make_map(reinterpret_cast<CUtensorMap*>(c->tc_map[0]), c->tc_Kf, 6LL * n, c->tc_ld,
                  c->tc_ld, kTcM) ||
        !make_map(reinterpret_cast<CUtensorMap*>(c->tc_map[1]), c->tc_V, (long long)vrows,
                  c->tc_ld, c->tc_ld, kTcNT) ||
        !make_map(reinterpret_cast<CUtensorMap*>(c->tc_map[2]), c->tc_V, (long long)vrows,
                  c->tc_ld, c->tc_ld, kTcN3))
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_tc_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTcSmem);
}

void tc_free(qdse_ctx* c) {
    for (float** p : {&c->tc_Kf, &c->tc_Kn, &c->tc_V}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
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
    const long long total = (long long)c->tc_nbt * kTcB * c->tc_ld;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    k_tc_prep<<<blocks, 256, 0, c->stream>>>(c->d_inst, c->work, c->tc_V, c->tc_n, c->n_inst,
                                             c->tc_nbt, c->tc_ld);
    TcArgs a{c->d_inst, c->d_state, c->grid.gdesc, c->grid, c->work, c->tc_Kn,
             c->tc_n, c->n_inst, c->n_total, c->tc_nbt, c->d_err};
    const dim3 grid((c->tc_n + kTcM - 1) / kTcM, c->tc_nbt);
    k_tc_sweep<<<grid, 128, kTcSmem, c->stream>>>(
        *reinterpret_cast<const CUtensorMap*>(c->tc_map[0]),
        *reinterpret_cast<const CUtensorMap*>(c->tc_map[1]),
        *reinterpret_cast<const CUtensorMap*>(c->tc_map[2]), a);
    c->launches += 2;
    prof_end(c);
    return cudaGetLastError();
}

}  // namespace qdse
