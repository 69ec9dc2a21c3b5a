// noalloc.cu -- one FP64 sweep of a single instance that allocates no memory at all.
//
// Some callers cannot allocate device memory. Examples: code running where the allocator is off
// limits (inside another library's memory pool or arena with a fixed budget, a real-time loop that
// must not call cudaMalloc/cudaFree because they synchronise the device, or an embedding that
// owns every byte of device memory itself).  For them qdse_sweep_fp64_noalloc evaluates the map
// x -> F(x) of the gap equation for one instance, in FP64 with the full (j, theta) double sum,
// using only the caller's input and output arrays and a fixed scratch array compiled into the
// library.
//
// The scratch is the file-scope array g_noalloc_scratch below (kNoallocDoubles doubles = 128 KB on
// every GPU that loads the library, kept until the process exits).  Host code cannot use the
// array's name as a device address: on the first call on each device (with that device current)
// the entry point asks the runtime for the address with cudaGetSymbolAddress and caches it per
// device.  Every call rebuilds all the scratch it reads (grid nodes, weights, stencil, node
// values) before reading it, so nothing depends on a previous call's contents.  All calls share
// the one array: calls whose work overlaps on the GPU (two streams, or two host threads) race on it
// and must be serialised by the caller.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "qdse_internal.h"

namespace qdse {
namespace {

constexpr int kNoallocMaxN = 512;
constexpr int kNoallocMaxTheta = 256;
// scratch: 11 per radial point (s_p, s_q, W, sqrt s_p, sqrt s_q, wt, 3 stencil coefficients, stencil
// start, u = ln s_p) + 4 per angular node + 4 per point (a, b at q, dA/ds, dB/ds)
constexpr int kNoallocDoubles = 16384;
static_assert(15 * kNoallocMaxN + 4 * kNoallocMaxTheta <= kNoallocDoubles, "scratch too small");

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

// Device address of g_noalloc_scratch per device index, looked up on the first call on that
// device.  Atomic slots: concurrent first calls from several host threads store the same value.
// A cudaDeviceReset unloads the module, so the address may change afterwards: the cache is not
// valid across a reset (documented at the declaration in qdse.h).
constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_ptr[kMaxDevices];

// Legendre P_n and P_n' by the three-term recurrence.
__device__ void na_legendre(int n, double x, double& p, double& dp) {
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    dp = n * (p0 - x * p1) / (1.0 - x * x);
}

struct NaLayout {
    double *sp, *sq, *W, *rsp, *rsq, *wt, *stc, *sta, *up, *z, *y, *s2, *wz, *aq, *bq, *dA, *dB;
};

__device__ NaLayout na_layout(double* base, int n, int nt) {
    NaLayout L;
    double* p = base;
    L.sp = p; p += n;
    L.sq = p; p += n;
    L.W = p; p += n;
    L.rsp = p; p += n;
    L.rsq = p; p += n;
    L.wt = p; p += n;
    L.stc = p; p += 3 * n;
    L.sta = p; p += n;
    L.up = p; p += n;
    L.z = p; p += nt;
    L.y = p; p += nt;
    L.s2 = p; p += nt;
    L.wz = p; p += nt;
    L.aq = p; p += n;
    L.bq = p; p += n;
    L.dA = p; p += n;
    L.dB = p; p += n;
    return L;
}

// Grid (log-mapped Gauss-Legendre radial rule, collocated or staggered; Gauss-Chebyshev angles),
// interpolated node values and the diagonal stencil quotients.  One block of kNoallocMaxN threads.
__global__ void __launch_bounds__(kNoallocMaxN) k_na_setup(double* scratch, qdse_grid gr,
                                                           const double* A, const double* B) {
    const int n = gr.n_p, nt = gr.n_theta, i = threadIdx.x;
    const NaLayout L = na_layout(scratch, n, nt);
    const double u0 = log(gr.s_min), u1 = log(gr.s_max);
    const double h = 0.5 * (u1 - u0), c = 0.5 * (u1 + u0);
    if (i < n) {
        // node i counted from x = -1 upwards: root k = n - i from the top, Newton from Tricomi
        const int k = n - i;
        double x = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) *
                   cos(kPi * (4.0 * k - 1.0) / (4.0 * n + 2.0));
        double p = 0.0, dp = 1.0;
        for (int it = 0; it < 50; ++it) {
            na_legendre(n, x, p, dp);
            const double dx = p / dp;
            x -= dx;
            if (fabs(dx) <= 1e-17) break;
        }
        na_legendre(n, x, p, dp);
        if (n % 2 == 1 && i == n / 2) x = 0.0;
        const double v = 2.0 / ((1.0 - x * x) * dp * dp);
        const double uq = c + h * x;
        L.sq[i] = exp(uq);
        L.W[i] = h * v * L.sq[i] * L.sq[i];
        L.up[i] = uq;  // staggered points are set below from neighbouring u
    }
    for (int kk = i; kk < nt; kk += blockDim.x) {
        const double th = (kk + 1) * kPi / (nt + 1);
        const double sn = sin(th), sh = sin(0.5 * th);
        L.z[kk] = cos(th);
        L.y[kk] = 2.0 * sh * sh;
        L.s2[kk] = sn * sn;
        L.wz[kk] = kPi / (nt + 1) * sn * sn;
    }
    __syncthreads();
    double upi = 0.0;
    if (i < n) {
        if (gr.grid_mode == QDSE_STAGGERED) upi = (i == 0) ? u0 : 0.5 * (L.up[i - 1] + L.up[i]);
        else upi = L.up[i];
    }
    __syncthreads();
    if (i < n) {
        L.up[i] = upi;
        L.sp[i] = (gr.grid_mode == QDSE_STAGGERED && i == 0) ? gr.s_min : exp(upi);
        if (gr.grid_mode == QDSE_COLLOCATED) L.sp[i] = L.sq[i];
        L.rsp[i] = sqrt(L.sp[i]);
        L.rsq[i] = sqrt(L.sq[i]);
    }
    __syncthreads();
    if (i < n) {
        if (gr.grid_mode == QDSE_STAGGERED && i < n - 1)
            L.wt[i] = (L.rsq[i] - L.rsp[i]) / (L.rsp[i + 1] - L.rsp[i]);
        else
            L.wt[i] = 0.0;
        int a = i - 1;
        if (a < 0) a = 0;
        if (a > n - 3) a = n - 3;
        const double x0 = L.up[a], x1 = L.up[a + 1], x2 = L.up[a + 2], x = L.up[i];
        L.stc[3 * i + 0] = ((x - x1) + (x - x2)) / ((x0 - x1) * (x0 - x2)) / L.sp[i];
        L.stc[3 * i + 1] = ((x - x0) + (x - x2)) / ((x1 - x0) * (x1 - x2)) / L.sp[i];
        L.stc[3 * i + 2] = ((x - x0) + (x - x1)) / ((x2 - x0) * (x2 - x1)) / L.sp[i];
        L.sta[i] = (double)a;
        // node values at q_i and the diagonal quotients
        double aq = A[i], bq = B[i];
        if (L.wt[i] != 0.0) {
            aq += L.wt[i] * (A[i + 1] - aq);
            bq += L.wt[i] * (B[i + 1] - bq);
        }
        L.aq[i] = aq;
        L.bq[i] = bq;
        L.dA[i] = L.stc[3 * i] * A[a] + L.stc[3 * i + 1] * A[a + 1] + L.stc[3 * i + 2] * A[a + 2];
        L.dB[i] = L.stc[3 * i] * B[a] + L.stc[3 * i + 1] * B[a + 1] + L.stc[3 * i + 2] * B[a + 2];
    }
}

// The sweep row i: the full double sum over (j, theta) of Eqs. dsesys/dsesys2 after the traces.
__global__ void __launch_bounds__(128) k_na_sweep(const double* scratch, qdse_grid gr,
                                                  qdse_params prm, int vertex, double kappa,
                                                  const double* A, const double* B, double* FA,
                                                  double* FB) {
    __shared__ double red[2][4];
    const int n = gr.n_p, nt = gr.n_theta, i = blockIdx.x;
    const NaLayout L = na_layout(const_cast<double*>(scratch), n, nt);
    const double P = L.sp[i], rP = L.rsp[i], Ai = A[i], Bi = B[i];
    const double iw2 = 1.0 / (prm.omega * prm.omega);
    const double pref = 8.0 * kPi * kPi * prm.D / (prm.omega * prm.omega * prm.omega * prm.omega);
    double sA = 0.0, sB = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double a = L.aq[j], bq = L.bq[j], Q = L.sq[j], rQ = L.rsq[j];
        const double e = L.W[j] / (Q * a * a + bq * bq);
        double qA, qB;
        if (gr.grid_mode == QDSE_COLLOCATED && j == i) {
            qA = L.dA[i];
            qB = L.dB[i];
        } else {
            qA = (a - Ai) / (Q - P);
            qB = (bq - Bi) / (Q - P);
        }
        const double SA = 0.5 * (Ai + a);
        const double dd = (rP - rQ) * (rP - rQ), c2 = 2.0 * rP * rQ, x0 = rP * rQ;
        const double PQ = P * Q, PpQ = P + Q;
        double S0 = 0.0, ST = 0.0, S3 = 0.0;
        for (int k = 0; k < nt; ++k) {
            const double k2 = dd + c2 * L.y[k];
            const double E = L.wz[k] * exp(-k2 * iw2);
            const double rk = 1.0 / k2;
            const double x = x0 * L.z[k];
            S0 += E;
            ST += E * 2.0 * PQ * L.s2[k] * rk;
            S3 += E * (3.0 * x * PpQ - 4.0 * x * x - 2.0 * PQ) * rk;
        }
        if (vertex == QDSE_VERTEX_BC) {
            sA += e * ((-bq * qB - 0.5 * PpQ * a * qA) * ST + a * SA * S3);
            sB += e * ((-a * qB + bq * qA) * ST + 3.0 * bq * SA * S0);
        } else {
            sA += e * a * S3;
            sB += 3.0 * e * bq * S0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sA += __shfl_xor_sync(0xffffffffu, sA, o);
        sB += __shfl_xor_sync(0xffffffffu, sB, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = sA;
        red[1][w] = sB;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double tA = red[0][0] + red[0][1] + red[0][2] + red[0][3];
        const double tB = red[1][0] + red[1][1] + red[1][2] + red[1][3];
        FA[i] = 1.0 + kappa * pref * tA / P;
        FB[i] = prm.m + kappa * pref * tB;
    }
}

void na_error(char* buf, int len, const char* msg) {
    if (buf && len > 0) {
        std::strncpy(buf, msg, (size_t)len - 1);
        buf[len - 1] = '\0';
    }
}

}  // namespace
}  // namespace qdse

using namespace qdse;

extern "C" qdse_status qdse_sweep_fp64_noalloc(const qdse_grid* g, const qdse_params* p,
                                               int vertex, double cf, const double* A,
                                               const double* B, double* FA, double* FB,
                                               void* stream, char* errbuf, int errbuf_len) {
    if (!g || !p || !A || !B || !FA || !FB) {
        na_error(errbuf, errbuf_len, "qdse_sweep_fp64_noalloc: null pointer argument");
        return QDSE_ERR_ARG;
    }
    if (g->n_p < 3 || g->n_p > kNoallocMaxN || g->n_theta < 1 || g->n_theta > kNoallocMaxTheta) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "qdse_sweep_fp64_noalloc: needs 3 <= n_p <= %d and 1 <= n_theta <= %d "
                      "(got n_p = %d, n_theta = %d)",
                      kNoallocMaxN, kNoallocMaxTheta, g->n_p, g->n_theta);
        na_error(errbuf, errbuf_len, msg);
        return QDSE_ERR_ARG;
    }
    if (!(g->s_min > 0.0) || !(g->s_max > g->s_min) || !std::isfinite(g->s_max) ||
        (g->grid_mode != QDSE_COLLOCATED && g->grid_mode != QDSE_STAGGERED) ||
        (vertex != QDSE_VERTEX_BC && vertex != QDSE_VERTEX_RL) || !(cf > 0.0) ||
        !std::isfinite(cf) || !std::isfinite(p->D) || p->D < 0.0 || !(p->omega > 0.0) ||
        !std::isfinite(p->omega) || !std::isfinite(p->m) || p->mu != 0.0) {
        na_error(errbuf, errbuf_len,
                 "qdse_sweep_fp64_noalloc: invalid grid, vertex, colour factor or parameters "
                 "(mu must be 0)");
        return QDSE_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        na_error(errbuf, errbuf_len, "qdse_sweep_fp64_noalloc: no usable current device");
        return QDSE_ERR_CUDA;
    }
    void* cached = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!cached) {
        // first call on this device: look up the device address of the scratch array
        e = cudaGetSymbolAddress(&cached, g_noalloc_scratch);
        if (e != cudaSuccess || !cached) {
            na_error(errbuf, errbuf_len, "qdse_sweep_fp64_noalloc: cudaGetSymbolAddress failed");
            return QDSE_ERR_CUDA;
        }
        g_scratch_ptr[dev].store(cached, std::memory_order_release);
    }
    double* scratch = static_cast<double*>(cached);
    cudaStream_t s = (cudaStream_t)stream;
    k_na_setup<<<1, kNoallocMaxN, 0, s>>>(scratch, *g, A, B);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_na_sweep<<<g->n_p, 128, 0, s>>>(scratch, *g, *p, vertex, cf / (8.0 * kPi * kPi * kPi),
                                          A, B, FA, FB);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "qdse_sweep_fp64_noalloc: launch failed: %s",
                      cudaGetErrorString(e));
        na_error(errbuf, errbuf_len, msg);
        return QDSE_ERR_CUDA;
    }
    na_error(errbuf, errbuf_len, "");
    return QDSE_OK;
}
