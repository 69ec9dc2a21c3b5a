// k_sweep_tma.cu -- the batched FP32 sweep (and its tangent) streamed through shared memory with
// bulk asynchronous copies (cp.async.bulk + mbarrier) by a producer warp.
//
// Work: for every external point p_i of every unfinished instance, the BC pair sums over the
// nonzero band of internal nodes j (Eqs. dsesys, dsesys2 after the traces; the pair formulas are in
// the header of k_sweep.cu).  The unit of scheduling is an item of up to rb consecutive rows of
// one instance; the update kernel of the previous tick lists the items of the instances that are
// still running.  A resident block (one per SM) takes items from that list with an atomic
// counter.  Per block:
//   warp 8 (producer) publishes each item's descriptor in shared memory, bulk-copies the
//     instance's node vectors (a, b, u1, u2, u3 and, for tangent sweeps, their directions) into one
//     of two vector buffers, and streams the kernel rows: every stage holds kStageRows rows, each
//     row's three planes copied over its nonzero band [jlo, jhi) only;
//   warps 0..7 (consumers) take one row of each stage, read it and the vectors from shared memory
//     with 16-byte conflict-free loads, reduce over the warp and write F (or J delta) for the row.
// Full/empty mbarriers order the stages, full/empty mbarriers the vector buffers.  Items of an
// instance in an FP64 phase are evaluated by the consumers straight from global memory.
//
// Every wait is bounded by a clock budget; on expiry the thread records an error flag (the host
// reports QDSE_ERR_TIMEOUT), and the block gives up its remaining work.
#include "qdse_internal.h"

namespace qdse {

constexpr int kConsumers = 8;            // consumer warps per block
constexpr int kStageRows = kConsumers;   // kernel rows per stage (one per consumer warp)
constexpr int kStagesT = 3;              // stages in the ring
constexpr int kMaxLdTma = 512;           // widest row this kernel handles
constexpr long long kWaitBudget = 4000000000LL;  // clock cycles (about 2 s)

struct ItemDesc {    // published by the producer for the consumers
    int b, row0, nrows, phase;
};

struct TmaLayout {
    int ldmax;
    size_t ring_floats, vec_floats;
    __host__ __device__ size_t bytes() const {
        return (ring_floats + 2 * vec_floats) * sizeof(float) +
               (2 * kStagesT + 4) * sizeof(unsigned long long) + 2 * sizeof(ItemDesc) +
               kStagesT * kStageRows * sizeof(int2);
    }
};

__host__ __device__ static TmaLayout tma_layout(int ldmax) {
    TmaLayout L;
    L.ldmax = ldmax;
    L.ring_floats = (size_t)kStagesT * kStageRows * 3 * ldmax;
    L.vec_floats = (size_t)10 * ldmax;
    return L;
}

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mb_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mb_expect(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mb_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mb_test(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mb_wait(unsigned long long* bar, uint32_t parity) {
    if (mb_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mb_test(bar, parity)) {
        if (clock64() - t0 > kWaitBudget) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void pairf(float a, float b, float u1, float u2, float u3, float K0,
                                      float KT, float K3, float Ai, float Bi, float Pi,
                                      float& sA, float& sB) {
    const float da = a - Ai, db = b - Bi, sa = Ai + a;
    const float cT = fmaf(-u1, db, -0.5f * fmaf(Pi, u2, u3) * da);
    sA = fmaf(cT, KT, fmaf(0.5f * u2 * sa, K3, sA));
    sB = fmaf(fmaf(u1, da, -u2 * db), KT, fmaf(1.5f * u1 * sa, K0, sB));
}

__device__ __forceinline__ void tpairf(float a, float b, float u1, float u2, float u3, float ea,
                                       float eb, float e1, float e2, float e3, float K0,
                                       float KT, float K3, float Ai, float Bi, float dAi,
                                       float dBi, float Pi, float& sA, float& sB) {
    const float da = a - Ai, db = b - Bi, sa = Ai + a;
    const float dda = ea - dAi, ddb = eb - dBi, dsa = dAi + ea;
    const float t = fmaf(Pi, u2, u3), dt = fmaf(Pi, e2, e3);
    const float dcT = -e1 * db - u1 * ddb - 0.5f * (dt * da + t * dda);
    sA = fmaf(dcT, KT, fmaf(0.5f * fmaf(e2, sa, u2 * dsa), K3, sA));
    sB = fmaf(e1 * da + u1 * dda - e2 * db - u2 * ddb, KT,
              fmaf(1.5f * fmaf(e1, sa, u1 * dsa), K0, sB));
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One FP64-phase row (residual or FP64 sweep on the double-float kernels), one warp.
__device__ void row64(int lane, const DevInst& I, int i, const Grid& g, const Work& w, int ntot,
                      const float* __restrict__ Khi, const float* __restrict__ Klo,
                      const double* A, const double* B, int vertex, double scale) {
    const int r = I.x_off + i;
    const int2 bd = g.band[r];
    const int jhi = min(bd.y, I.n);
    const long long plane = I.ld;  // planes of a row are adjacent
    const long long row = I.k_off + (long long)i * 3 * I.ld;
    const double* v = w.vec64;
    const double Ai = A[r], Bi = B[r], P = g.sp[r];
    double sA = 0.0, sB = 0.0;
    for (int j = bd.x + lane; j < jhi; j += 32) {
        const int gj = I.x_off + j;
        const double K0 = (double)Khi[row + j] + (double)Klo[row + j];
        const double KT = (double)Khi[row + plane + j] + (double)Klo[row + plane + j];
        const double K3 = (double)Khi[row + 2 * plane + j] + (double)Klo[row + 2 * plane + j];
        const double a = v[gj], b = v[ntot + gj], u1 = v[2 * ntot + gj], u2 = v[3 * ntot + gj],
                     u3 = v[4 * ntot + gj];
        if (vertex == QDSE_VERTEX_BC) {
            const double da = a - Ai, db = b - Bi, sa = Ai + a;
            sA += (-u1 * db - 0.5 * (P * u2 + u3) * da) * KT + 0.5 * u2 * sa * K3;
            sB += (u1 * da - u2 * db) * KT + 1.5 * u1 * sa * K0;
        } else {
            sA += u2 * K3;
            sB += 3.0 * u1 * K0;
        }
    }
    sA = wsum(sA);
    sB = wsum(sB);
    if (lane == 0) {
        if (vertex == QDSE_VERTEX_BC && I.mode == QDSE_COLLOCATED) {
            const double KTd = (double)Khi[row + plane + i] + (double)Klo[row + plane + i];
            const double dA = w.dia64[r], dB = w.dia64[ntot + r];
            sA += (-v[2 * ntot + r] * dB - P * v[3 * ntot + r] * dA) * KTd;
            sB += (v[2 * ntot + r] * dA - v[3 * ntot + r] * dB) * KTd;
        }
        w.xn64[r] = 1.0 + scale * sA / P;
        w.xn64[ntot + r] = I.m + scale * sB;
    }
}

__global__ void __launch_bounds__((kConsumers + 1) * 32, 1) k_sweep_items(
    const DevInst* __restrict__ inst, const DevState* __restrict__ state,
    const Ctl* __restrict__ ctl, Grid g, Work w, const float* __restrict__ Khi,
    const float* __restrict__ Klo, const double* A, const double* B, int ntot, int buf,
    int ldmax, int* err_flag) {
    extern __shared__ __align__(128) unsigned char smem[];
    const TmaLayout L = tma_layout(ldmax);
    float* ring = reinterpret_cast<float*>(smem);
    float* vbuf = ring + L.ring_floats;  // [2][10][ldmax]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(vbuf + 2 * L.vec_floats);
    unsigned long long* full = bars;                  // [kStagesT]
    unsigned long long* empty = bars + kStagesT;      // [kStagesT]
    unsigned long long* vfull = bars + 2 * kStagesT;  // [2]
    unsigned long long* vempty = vfull + 2;           // [2]
    ItemDesc* desc = reinterpret_cast<ItemDesc*>(vempty + 2);      // [2]
    int2* sband = reinterpret_cast<int2*>(desc + 2);               // [kStagesT][kStageRows]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesT; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], kConsumers);
        }
        for (int k = 0; k < 2; ++k) {
            mb_init(&vfull[k], 1);
            mb_init(&vempty[k], kConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (blockIdx.x == 0) w.item_count[buf ^ 1] = 0;  // the next tick's list is rebuilt
    }
    __syncthreads();

    const int nitems = w.item_count[buf];
    const int2* items = w.items + (size_t)buf * w.max_items;
    const int vertex = ctl->vertex;
    const int nv = w.nv;

    if (warp == kConsumers) {
        // ------------------------------------------------------------------ producer warp
        long long q = 0;  // stages issued so far (global over items)
        int k = 0;        // items taken so far
        bool ok = true;
        while (ok) {
            int it = 0;
            if (lane == 0) it = atomicAdd(w.work_ctr, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            const int vb = k & 1;
            if (k >= 2 && !mb_wait(&vempty[vb], ((k >> 1) - 1) & 1)) { ok = false; break; }
            if (it >= nitems) {
                if (lane == 0) {
                    desc[vb].b = -1;
                    mb_arrive(&vfull[vb]);
                }
                break;
            }
            const int2 item = items[it];
            const DevInst I = inst[item.x];
            const int phase = state[item.x].phase;
            const int row0 = item.y, nrows = min(w.rb, I.n - item.y);
            const bool tan = (phase == PH_TANGENT32);
            const bool f32 = (phase == PH_PICARD32) || tan;
            if (lane == 0) {
                desc[vb].b = item.x;
                desc[vb].row0 = row0;
                desc[vb].nrows = nrows;
                desc[vb].phase = phase;
            }
            // node vectors of the instance (whole padded row: ld floats per component)
            const uint32_t vbytes = (uint32_t)I.ld * 4u;
            const int nvec = f32 ? (tan ? 10 : 5) : 0;
            __syncwarp();
            if (lane == 0) {
                if (nvec) mb_expect(&vfull[vb], vbytes * (uint32_t)nvec);
                else mb_arrive(&vfull[vb]);
            }
            __syncwarp();
            if (lane < nvec) {
                const float* base = (lane < 5) ? w.vec32 : w.dvec32;
                bulk_g2s(vbuf + (size_t)vb * L.vec_floats + (size_t)lane * ldmax,
                         base + (size_t)(lane % 5) * nv + I.v_off, vbytes, &vfull[vb]);
            }
            ++k;
            if (!f32) continue;
            // kernel rows, kStageRows per stage, each over its own band
            const long long plane = I.ld;  // planes of a row are adjacent
            for (int r0 = 0; r0 < nrows && ok; r0 += kStageRows) {
                const int s = (int)(q % kStagesT);
                if (q >= kStagesT && !mb_wait(&empty[s], (uint32_t)(((q / kStagesT) - 1) & 1))) {
                    ok = false;
                    break;
                }
                const int rr = r0 + lane;
                int2 bd = make_int2(0, 0);
                if (lane < kStageRows && rr < nrows) bd = g.band[I.x_off + row0 + rr];
                if (lane < kStageRows) sband[s * kStageRows + lane] = bd;
                uint32_t bytes = (uint32_t)(bd.y - bd.x) * 12u;
                bytes = wsum(bytes);
                __syncwarp();
                if (lane == 0) mb_expect(&full[s], bytes);
                __syncwarp();
                if (lane < kStageRows && bd.y > bd.x) {
                    const int i = row0 + rr;
                    const uint32_t seg = (uint32_t)(bd.y - bd.x) * 4u;
                    float* dst = ring + ((size_t)s * kStageRows + lane) * 3 * ldmax + bd.x;
                    const float* src = Khi + I.k_off + (long long)i * 3 * I.ld + bd.x;
                    bulk_g2s(dst, src, seg, &full[s]);
                    bulk_g2s(dst + ldmax, src + plane, seg, &full[s]);
                    bulk_g2s(dst + 2 * ldmax, src + 2 * plane, seg, &full[s]);
                }
                ++q;
            }
        }
        if (!ok && lane == 0) atomicExch(err_flag, 1);
        return;
    }

    // ---------------------------------------------------------------------- consumer warps
    long long q = 0;
    int k = 0;
    while (true) {
        const int vb = k & 1;
        if (!mb_wait(&vfull[vb], (k >> 1) & 1)) {
            if (lane == 0) atomicExch(err_flag, 1);
            return;
        }
        const ItemDesc d = desc[vb];
        if (d.b < 0) return;
        const DevInst I = inst[d.b];
        const double scale = ctl->kappa * I.D;
        const bool tan = (d.phase == PH_TANGENT32);
        const bool f32 = (d.phase == PH_PICARD32) || tan;
        if (!f32) {
            for (int rr = warp; rr < d.nrows; rr += kConsumers)
                row64(lane, I, d.row0 + rr, g, w, ntot, Khi, Klo, A, B, vertex, scale);
        } else {
            const float* V = vbuf + (size_t)vb * L.vec_floats;
            for (int r0 = 0; r0 < d.nrows; r0 += kStageRows) {
                const int s = (int)(q % kStagesT);
                const int rr = r0 + warp;
                const bool valid = rr < d.nrows;
                const int i = d.row0 + rr, gi = I.x_off + i;
                // own values and diagonal data of this row (loads overlap the wait)
                float Ai = 0.f, Bi = 0.f, Pi = 0.f, dAi = 0.f, dBi = 0.f;
                if (valid) {
                    Ai = w.x32[gi];
                    Bi = w.x32[ntot + gi];
                    Pi = g.sp32[gi];
                    if (tan) {
                        dAi = w.d32[gi];
                        dBi = w.d32[ntot + gi];
                    }
                }
                if (!mb_wait(&full[s], (uint32_t)((q / kStagesT) & 1))) {
                    if (lane == 0) atomicExch(err_flag, 1);
                    return;
                }
                float sA = 0.f, sB = 0.f;
                if (valid) {
                    const int2 bd = sband[s * kStageRows + warp];
                    const float* Kr = ring + ((size_t)s * kStageRows + warp) * 3 * ldmax;
                    for (int c = bd.x + 4 * lane; c < bd.y; c += 128) {
                        const float4 K0 = *reinterpret_cast<const float4*>(Kr + c);
                        const float4 KT = *reinterpret_cast<const float4*>(Kr + ldmax + c);
                        const float4 K3 = *reinterpret_cast<const float4*>(Kr + 2 * ldmax + c);
                        const float4 a = *reinterpret_cast<const float4*>(V + c);
                        const float4 b = *reinterpret_cast<const float4*>(V + ldmax + c);
                        const float4 u1 = *reinterpret_cast<const float4*>(V + 2 * ldmax + c);
                        const float4 u2 = *reinterpret_cast<const float4*>(V + 3 * ldmax + c);
                        const float4 u3 = *reinterpret_cast<const float4*>(V + 4 * ldmax + c);
                        if (vertex == QDSE_VERTEX_BC) {
                            if (!tan) {
                                pairf(a.x, b.x, u1.x, u2.x, u3.x, K0.x, KT.x, K3.x, Ai, Bi, Pi, sA, sB);
                                pairf(a.y, b.y, u1.y, u2.y, u3.y, K0.y, KT.y, K3.y, Ai, Bi, Pi, sA, sB);
                                pairf(a.z, b.z, u1.z, u2.z, u3.z, K0.z, KT.z, K3.z, Ai, Bi, Pi, sA, sB);
                                pairf(a.w, b.w, u1.w, u2.w, u3.w, K0.w, KT.w, K3.w, Ai, Bi, Pi, sA, sB);
                            } else {
                                const float4 ea = *reinterpret_cast<const float4*>(V + 5 * ldmax + c);
                                const float4 eb = *reinterpret_cast<const float4*>(V + 6 * ldmax + c);
                                const float4 e1 = *reinterpret_cast<const float4*>(V + 7 * ldmax + c);
                                const float4 e2 = *reinterpret_cast<const float4*>(V + 8 * ldmax + c);
                                const float4 e3 = *reinterpret_cast<const float4*>(V + 9 * ldmax + c);
                                tpairf(a.x, b.x, u1.x, u2.x, u3.x, ea.x, eb.x, e1.x, e2.x, e3.x, K0.x, KT.x, K3.x, Ai, Bi, dAi, dBi, Pi, sA, sB);
                                tpairf(a.y, b.y, u1.y, u2.y, u3.y, ea.y, eb.y, e1.y, e2.y, e3.y, K0.y, KT.y, K3.y, Ai, Bi, dAi, dBi, Pi, sA, sB);
                                tpairf(a.z, b.z, u1.z, u2.z, u3.z, ea.z, eb.z, e1.z, e2.z, e3.z, K0.z, KT.z, K3.z, Ai, Bi, dAi, dBi, Pi, sA, sB);
                                tpairf(a.w, b.w, u1.w, u2.w, u3.w, ea.w, eb.w, e1.w, e2.w, e3.w, K0.w, KT.w, K3.w, Ai, Bi, dAi, dBi, Pi, sA, sB);
                            }
                        } else {
                            const float4 p2 = tan ? *reinterpret_cast<const float4*>(V + 8 * ldmax + c) : u2;
                            const float4 p1 = tan ? *reinterpret_cast<const float4*>(V + 7 * ldmax + c) : u1;
                            sA += p2.x * K3.x + p2.y * K3.y + p2.z * K3.z + p2.w * K3.w;
                            sB += 3.f * (p1.x * K0.x + p1.y * K0.y + p1.z * K0.z + p1.w * K0.w);
                        }
                    }
                }
                sA = wsum(sA);
                sB = wsum(sB);
                if (valid && lane == 0) {
                    if (vertex == QDSE_VERTEX_BC && I.mode == QDSE_COLLOCATED) {
                        const float* Kr = ring + ((size_t)s * kStageRows + warp) * 3 * ldmax;
                        const float KTd = Kr[ldmax + i];  // the diagonal lies in every band
                        const float u1 = V[2 * ldmax + i], u2 = V[3 * ldmax + i];
                        const float dA = w.dia32[gi], dB = w.dia32[ntot + gi];
                        if (!tan) {
                            sA += (-u1 * dB - Pi * u2 * dA) * KTd;
                            sB += (u1 * dA - u2 * dB) * KTd;
                        } else {
                            const float e1 = V[7 * ldmax + i], e2 = V[8 * ldmax + i];
                            const float edA = w.ddia32[gi], edB = w.ddia32[ntot + gi];
                            sA += (-e1 * dB - u1 * edB - Pi * (e2 * dA + u2 * edA)) * KTd;
                            sB += (e1 * dA + u1 * edA - e2 * dB - u2 * edB) * KTd;
                        }
                    }
                    if (!tan) {
                        w.xn32[gi] = (float)(1.0 + scale * (double)sA / g.sp[gi]);
                        w.xn32[ntot + gi] = (float)(I.m + scale * (double)sB);
                    } else {
                        w.xn32[gi] = (float)(scale * (double)sA / g.sp[gi]);
                        w.xn32[ntot + gi] = (float)(scale * (double)sB);
                    }
                }
                __syncwarp();
                if (lane == 0) mb_arrive(&empty[s]);
                ++q;
            }
        }
        __syncwarp();
        if (lane == 0) mb_arrive(&vempty[vb]);
        ++k;
    }
}

size_t sweep_items_smem_bytes(int ldmax) { return tma_layout(ldmax).bytes(); }

cudaError_t launch_sweep32_tma(qdse_ctx* c, const double* A, const double* B) {
    prof_begin(c, PK_SWEEP);
    k_sweep_items<<<c->n_sms, (kConsumers + 1) * 32, sweep_items_smem_bytes(c->ld_max),
                    c->stream>>>(c->d_inst, c->d_state, c->d_ctl, c->grid, c->work, c->d_Khi,
                                 c->d_Klo, A, B, c->n_total, c->tick & 1, c->ld_max, c->d_err);
    c->launches++;
    prof_end(c);
    return cudaGetLastError();
}

cudaError_t configure_sweep32_tma(int ldmax) {
    if (ldmax > kMaxLdTma) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_sweep_items, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_items_smem_bytes(ldmax));
}

}  // namespace qdse
