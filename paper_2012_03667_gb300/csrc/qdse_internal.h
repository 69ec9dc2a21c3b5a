// qdse_internal.h -- internal data structures of libqdse (not part of the C interface).
//
// Device memory layout (all arrays structure-of-arrays over the batch):
//   points      : every instance b owns global point indices [x_off[b], x_off[b] + n_b).
//                 FP64 grid arrays (s_p, s_q, W, ...) and every per-point work vector use this
//                 index; vectors with several components are stored component-major with stride
//                 n_total (component c of point g at [c * n_total + g]).
//   kernel pool : instance b owns n_b rows (external p_i) of 3 planes x ld_b floats starting at
//                 k_off[b]: entry (i, plane, j) at k_off + (3 i + plane) ld + j, plane 0 = K_0,
//                 1 = K_T / (Q_j - P_i) (diagonal: K_T), 2 = K_3, columns j (internal q_j),
//                 ld_b = n_b rounded up to 4 (the three planes of a row are adjacent).  The
//                 same layout holds the low parts (double-float residues) in a second buffer and,
//                 for the adjoint, the omega-derivatives of the three kernels.
//   angular     : instance b owns nodes [t_off[b], t_off[b] + n_theta_b).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qdse.h"

namespace qdse {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kMaxN = 1024;
constexpr int kMaxTheta = 512;

// Solver phases of one instance (a small state machine advanced on the device).
enum Phase : int {
    PH_PICARD32 = 0,  // FP32 successive approximation on the precomputed kernels
    PH_RESID64 = 1,   // FP64 evaluation of F(x) for the refinement residual
    PH_TANGENT32 = 2, // FP32 tangent sweep J(x) delta for the correction solve
    PH_PICARD64 = 3,  // FP64 successive approximation (precomputed or on-the-fly kernels)
    PH_DONE = 4
};

struct DevInst {          // per-instance descriptor, read-only during a solve
    int n;                // radial points
    int nt;               // angular nodes
    int x_off;            // first global point
    int t_off;            // first angular node
    long long k_off;      // first element of this instance's block of the kernel pool
    int ld;               // columns stored per kernel row (n rounded up to 4)
    int mode;             // QDSE_COLLOCATED / QDSE_STAGGERED
    int v_off;            // first node of this instance in the padded FP32 node vectors
    int g_off;            // first row group of this instance
    int s_off;            // first slab (kSlabGroups row groups) of this instance
    int pad;
    double D, omega, m;   // current parameters
};

struct GroupDesc {        // one row group (kRows consecutive external points of one instance)
    int b, i0, nr, jlo;   // instance, first row, rows in the group, band union start
    int jhi, v_off, x_off, ld;  // band union end, node-vector base, point base, kernel columns
    long long kbase;      // kernel-pool offset of the group's block (see kpos)
    int mode;             // grid mode of the instance
    float sc32, m32;      // kappa D and m of the instance in FP32 (refreshed with every
                          // parameter upload)
    int ng;               // row groups of the instance
    int pad[2];
};

constexpr int kSlabGroups = 8;  // row groups per slab (the slab sweep's unit of work: 32 rows)

struct SlabRec {          // one slab: up to kSlabGroups consecutive row groups of one instance
    int b, g0, ng, x_off;      // instance, first group, groups in the slab, the instance's first point
    int v_off, n, ld, mode;    // node-vector base, points, kernel columns, grid mode
    long long k_off;           // the instance's kernel-pool block
    float sc32, m32;           // kappa D and m in FP32 (refreshed with every parameter upload)
    int2 band[kSlabGroups];    // union band [jlo, jhi) of every group of the slab
    int pad[4];
};
static_assert(sizeof(SlabRec) == 128, "slab records are copied as eight 16-byte words");

struct DevState {         // per-instance solver state, updated by the update kernel
    int phase;
    int iters;            // sweeps of any kind
    int inner;            // tangent sweeps in the current correction solve
    int status;           // qdse_status of the instance
    double change;        // last R7 relative change (Picard) or residual
    double dnorm;         // last relative change of the correction (inner solve)
    int loc;              // 1 if the current iterate lives in the FP32 copy, 0 if in A, B
    int n64;              // FP64 sweeps (Picard and refinement residuals) of this solve
    float cbest;          // lowest relative change of the current Picard phase
    int since;            // Picard sweeps since cbest was set
    int stall_max;        // longest such run of this solve
    int nh;               // iterate hashes recorded in the current Picard phase
    unsigned long long href;  // cycle detection (Brent): the reference hash, recorded at hash
    int iref, plen;           // number iref; it moves after plen more hashes, plen doubling
    int cyc_p, cyc_at;        // period of a detected cycle and the sweep that found it (0: none)
};
constexpr int kHashRing = 16;  // recent iterate hashes per instance (cycles of period <= 16 are
                               // found one period after they start; longer ones by Brent's rule)

struct Ctl {              // solver controls shared by every instance of a call
    double kappa;         // C_F / (8 pi^3)
    double tol;           // final tolerance
    double sw_tol;        // FP32 -> refinement switch threshold
    double inner_tol;     // relative change that ends a correction solve
    double alpha;         // relaxation
    int max_iter;
    int max_inner;        // tangent sweeps per correction solve
    int max_fp32;         // cap of the FP32 Picard phase
    int vertex;           // QDSE_VERTEX_BC / _RL
    int precision;
    int final_phase;      // PH_PICARD64 for FP64 modes, PH_PICARD32 for FP32-only
    int never_converge;   // 1 for qdse_iterate (run exactly max_iter sweeps)
    int stall_copies;     // test of the bounded waits: the ring sweep expects 16 bytes more than
                          // it copies per tile, so each tile wait runs out (QDSE_TEST_STALL=1)
    int stall_window;     // no-progress stop of the Picard phases (0 = off)
    int stop_cycles;      // end a Picard phase whose iterate repeats exactly (0 = off)
    int slab_lists;       // 1: keep the slab lists and slab phases (the slab sweep reads them)
    int tc_picard;        // 1: FP32 Picard rows are swept by the tensor-core product (k_tc.cu),
                          // so instances in that phase put no row groups on the active lists
    int narrow_split;     // 1: full row groups of a Ball-Chiu FP32 Picard sweep whose band is at
                          // most kNarrowCols columns go on the narrow list (k_tick_narrow), the
                          // others on the group list (the ring sweep)
};

// Work arrays (device).  Component counts in brackets, each of length n_total.
struct Work {
    double* xn64;   // [2] F(x) in FP64 (residual / FP64 sweeps)
    double* r64;    // [2] refinement right-hand side r = F(x) - x
    double* d64;    // [2] correction delta (FP64 master)
    double* vec64;  // [5] per internal node: a, b, u1 = e b, u2 = e a, u3 = e a Q (FP64)
    double* dia64;  // [2] diagonal difference quotients dA/ds, dB/ds at p_i (collocated)
    int nv;         // length of one component of vec32 / dvec32 (sum of ld, multiple of 4)
    float* x32;     // [2] FP32 iterate
    float* xn32;    // [2] FP32 sweep output (F(x) or J delta)
    float* vec32;   // [5] FP32 copies of vec64 entries at the current iterate, padded layout:
                    //     component c of node j of instance b at [c * nv + v_off_b + j], zero in
                    //     the padding so that 16-byte loads of 4 nodes stay aligned
    float* dia32;   // [2]
    float* dvec32;  // [5] tangent: delta a, delta b, delta u1, delta u2, delta u3 (padded layout)
    float* ddia32;  // [2] tangent: stencil of delta
    float* d32;     // [2] FP32 copy of the correction (delta A_i, delta B_i at p_i)
    double* dvec64; // [5] FP64 tangent vectors (Jacobian-vector products)
    double* ddia64; // [2]
    double* lam;    // [2] adjoint iterate
    double* lamn;   // [2] adjoint sweep output
    // active lists: instances, row groups and slabs still running, three buffers (tick t reads
    // list t % 3, appends the survivors to (t + 1) % 3 and empties (t + 2) % 3);
    // lcount = {instances[0..2], groups[0..2], slabs[0..2], narrow groups[0..2]}
    int* ilist;     // [3][n_inst]
    int* glist;     // [3][n_groups]
    int* lcount;    // [12]: instances, groups, slabs, narrow groups (three buffers each)
    int* nlist;     // [3][n_groups] narrow row groups (Ctl::narrow_split)
    int* slist;     // [3][n_slabs] active slabs (same three-buffer scheme)
    int* sphase;    // [n_slabs] the phase of the slab's instance for the coming sweep
    int* claim;     // [3] slab claims of the tick that reads list t % 3 (the slab sweep)
    int n_slabs;
    unsigned long long* hring;  // [n_inst][kHashRing] recent iterate hashes (cycle detection)
    int* ticket;    // [n_inst] row groups of the instance swept in the current tick (the fused
                    // update: the warp that completes the last one advances the instance)
    double* col;    // [2] transposed sweep on staggered grids: per internal node, the summed
                    // derivatives through its interpolated values
    int n_inst;
    int n_groups;
};

struct Grid {              // FP64 grid arrays on the device (global point index)
    double* sp;            // external nodes s_p = p^2
    double* sq;            // internal nodes s_q = q^2
    double* W;             // internal weights, int ds s f ~ sum W f
    double* rsp;           // sqrt(s_p)
    double* rsq;           // sqrt(s_q)
    double* wt;            // staggered: weight of the upper bracket point (0 at the last node)
    double* stc;           // [3] collocated: Lagrange derivative coefficients (per s) of the stencil
    int* sta;              // collocated: first point of the stencil (local index)
    float* sp32;           // float copies (for the FP32 sweeps and their updates)
    float* sq32;
    float* W32;
    float* wt32;
    float* stc32;          // [3]
    double* z;             // angular nodes (per instance slice)
    double* y;             // 1 - z
    double* s2;            // 1 - z^2
    double* wz;            // angular weights
    int* row_inst;         // instance of every global point
    int2* band;            // per external point: [jlo, jhi) outside which every kernel entry of
                           // the row is exactly zero (jlo, jhi multiples of 4, jhi <= ld)
    int2* groups;          // (instance, first row) of every group of kRows consecutive rows
    struct GroupDesc* gdesc;  // per group: everything a sweep needs to start its loads
    int* gphase;           // per group: the phase of its instance for the coming sweep
    unsigned long long* nnz;  // per instance: sum over rows of the band widths (kernel entries a
                              // sweep must read per plane)
    int* nfirst;           // per instance: the first row group from which every full group up to
                           // the last full one is narrow (band of at most kNarrowCols columns)
    float* ktd;            // per external point: K_T at q = p (collocated grids; the entry the
                           // removable-limit term multiplies), 0 on staggered grids
    struct SlabRec* slabs; // per slab: the slab sweep's record (bands refreshed with the kernels)
    float2* expt;          // exp(-a/4) and exp(-b/512) as (hi, lo) pairs for the FP32-pipe
                           // precompute (see k_precompute.cu)
};

constexpr int kTuneCandidates = 5;  // qdse_autotune: ring 12x2, 8x3, 6x4, slab, register-only
constexpr int kRows = 4;   // external points per warp in the batched sweeps (1, 2 or 4)
constexpr int kTickBlocksPerSM = kRows >= 4 ? 2 : 3;  // resident 256-thread sweep blocks per SM
constexpr int kTile = 32;  // kernel precompute tile edge
constexpr int kNarrowCols = 32;  // narrow row group: a band of at most this many columns
// Kernel pool layout.  The entries K_p(i, j) (plane p = 0, 1, 2 for K_0, K_T/(Q - P), K_3) of one
// instance fill n * 3 * ld floats from k_off.  Rows come in groups of kRows (the last group may be
// shorter, nr rows); a group's block starts at k_off + 3 i0 ld, and each 4-column block q of it
// stores the 3 nr plane-rows m = 3 r + p as consecutive float4.  So any column range of a group
// is one contiguous run (one bulk copy), and a lane reading one 4-column block gets all the
// group's rows from adjacent 16-byte words.  For full groups of 4 rows the 12 plane-rows of block
// q are stored in the order m ^ ((q >> 1) & 3), which makes 16-byte shared-memory reads of 8
// consecutive blocks hit 8 different bank quads.
__host__ __device__ inline int kswz(int nr, int q) {
    return ((3 * nr) & 3) == 0 ? ((q >> 1) & 3) : 0;
}
__host__ __device__ inline long long kpos(long long k_off, int n, int ld, int i, int p, int j) {
    const int i0 = i - i % kRows;
    const int nr = (n - i0 < kRows) ? n - i0 : kRows;
    const int m = 3 * (i - i0) + p, q = j >> 2;
    return k_off + 3LL * i0 * ld + ((long long)q * 3 * nr + (m ^ kswz(nr, q))) * 4 + (j & 3);
}
// FP32 node vectors (a, b, u1, u2, u3 and their tangents): component c of padded node x (= v_off
// + j) at 20 (x / 4) + 4 c + x % 4, so the five components of a 4-node block are one 80-byte run
// and any node range of an instance is contiguous.
__host__ __device__ inline long long vpos(int x, int c) {
    return 20LL * (x >> 2) + 4 * c + (x & 3);
}

struct HostInst {
    qdse_grid g;
    int x_off, t_off, ld, v_off, g_off, s_off;
    long long k_off;
};

#ifdef __CUDACC__
// Pool offsets of one kernel row i (see kpos): off(p, j) for plane p, column j.
struct KRow {
    long long base;  // the group's block
    int nr, m0;      // rows in the group, plane-row of (i, plane 0)
    __device__ KRow(const DevInst& I, int i) {
        const int i0 = i - i % kRows;
        base = I.k_off + 3LL * i0 * I.ld;
        nr = min(kRows, I.n - i0);
        m0 = 3 * (i - i0);
    }
    __device__ long long off(int p, int j) const {
        return base + ((long long)(j >> 2) * 3 * nr + ((m0 + p) ^ kswz(nr, j >> 2))) * 4 + (j & 3);
    }
};

// Warp sums of 2 kRows values at once (v[0..kRows) = A sums, v[kRows..2 kRows) = B sums of the
// group's rows): each butterfly step halves the values a lane carries, so the lane 32/(2 kRows) * q
// ends with the total of value q after (2 kRows - 1) + log2(32/(2 kRows)) shuffles.
__device__ __forceinline__ float group_totals(const float* sA, const float* sB, int lane) {
    constexpr int NV = 2 * kRows;
    float v[NV];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        v[r] = sA[r];
        v[kRows + r] = sB[r];
    }
    int width = NV;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        if (width > 1) {
            const bool hi = (lane & m) != 0;
            const int half = width >> 1;
#pragma unroll
            for (int k = 0; k < NV / 2; ++k) {
                if (k < half) {
                    const float keep = hi ? v[k + half] : v[k], send = hi ? v[k] : v[k + half];
                    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                }
            }
            width = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
        }
    }
    return v[0];
}
// index of the value whose total lane `lane` holds after group_totals
__device__ __forceinline__ int group_total_index(int lane) { return lane / (32 / (2 * kRows)); }
// lanes that hold a total first in their run
__device__ __forceinline__ bool group_total_leader(int lane) {
    return (lane % (32 / (2 * kRows))) == 0;
}
#endif

}  // namespace qdse

struct qdse_ctx {
    int n_inst = 0;
    int n_total = 0;
    int nv_total = 0;        // sum of ld (padded FP32 vector length)
    int n_groups = 0;        // row groups of kRows
    int n_slabs = 0;         // slabs of kSlabGroups row groups
    int t_total = 0;
    long long k_total = 0;   // floats per kernel plane set (sum of 3 n ld)
    int max_n = 0, max_nt = 0;
    qdse_options opt{};
    cudaStream_t stream = nullptr;
    std::vector<qdse::HostInst> hinst;
    std::vector<double> h_sp, h_sq, h_W;  // host copies of the grid
    bool any_staggered = false;

    qdse::DevInst* d_inst = nullptr;
    qdse::DevState* d_state = nullptr;
    qdse::Ctl* d_ctl = nullptr;
    qdse::Grid grid{};
    qdse::Work work{};
    float* d_Khi = nullptr;
    float* d_Klo = nullptr;
    float* d_Kwhi = nullptr;  // omega-derivative kernels (allocated on first adjoint)
    float* d_Kwlo = nullptr;
    int* d_count = nullptr;   // [2] unfinished instances after the last update; error flag
    unsigned long long* d_sweeps = nullptr;  // [4] FP32 / FP64 instance-sweeps, algorithmic
                                             // bytes of the sweeps, BC-kernel evaluations
    double* d_hostA = nullptr;  // staging for qdse_solve_host: [2 n_total] doubles
    int* d_hostI = nullptr;     // [2 n_inst] ints (iterations, status)
    int* h_count = nullptr;   // pinned mirror of d_count[0..1]
    int* d_err = nullptr;     // = d_count + 1: set when a bounded device wait ran out
    int n_sms = 0;
    int ld_max = 0;           // widest kernel row of the batch
    int sweep_kind = 0;       // FP32 sweep: 2 slab (bulk copies through shared memory, slabs of
                              // row groups), 1 ring (the same per row group), 0 register-only
    int precompute_kind = 1;  // kernel matrices: 1 double-float on the FP32 pipe (default), 0 FP64
    int ring_shape = 0;       // ring sweep: 0 = 12 warps x 2 slots, 1 = 8 x 3, 2 = 6 x 4
    int slab_ok = 0;          // the slab sweep could be configured on this device
    // shared kernels (options.shared_kernels): the tensor-core Picard sweep of k_tc.cu
    int tc = 0, tc_n = 0, tc_ld = 0, tc_bp = 0, tc_ldg = 0;
    float* tc_Kf = nullptr;   // [2][3 n][tc_ld] far-field planes, TF32 high and low parts
    float* tc_Kn = nullptr;   // [3][n][17] near band
    float* tc_V = nullptr;    // [2][11 tc_bp][tc_ld] column functions of the batch (TF32 parts)
    float* tc_G = nullptr;    // [11 tc_bp][tc_ldg] far-field products
    int* tc_any = nullptr;    // [tc_bp / 128] blocks of instances with one in the Picard phase
    alignas(64) unsigned char tc_map[2][128];  // tensor maps: column functions, kernel planes
    int narrow_ok = 1;        // the narrow list may be used (QDSE_NARROW=0 at creation turns it off)
    int fused_update = 0;     // ring sweep: 1 advances each instance inside the sweep launch (one
                              // launch per tick), 0 in a separate k_update launch (the default)
    int4* d_tiles = nullptr;  // precompute tiles (instance, tile row, tile column)
    double* d_rel = nullptr;  // [n_inst] relative residual of the adjoint's fixed point
    // CUDA graph of a chunk of ticks, replayed between polls (captured on an internal stream)
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const double* g_A = nullptr;
    const double* g_B = nullptr;
    int g_path = -1;
    long long g_launches = 0;  // kernels per replay
    int n_tiles = 0;
    long long tick = 0;       // ticks issued since the last init (selects the active-list buffers)
    qdse::DevInst* h_inst_pinned = nullptr;

    std::string err;
    long long launches = 0, sweeps32 = 0, sweeps64 = 0, polls = 0;
    // optional CUDA-event timing of every launch, by kind (see qdse::ProfKind)
    int profiling = 0;
    int stall_copies = 0;     // QDSE_TEST_STALL=1 at creation (see Ctl::stall_copies)
    struct ProfRec { int kind; cudaEvent_t a, b; };
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> prof;
    int k_valid_for = 0;     // 1 if the kernel pool matches the parameters in d_inst (w, grid)
    int kw_valid = 0;
    std::vector<double> k_omega;  // omega each instance's kernels were built for
};

namespace qdse {

enum ProfKind : int { PK_PRECOMPUTE = 0, PK_SWEEP = 1, PK_UPDATE = 2, PK_OTHER = 3, PK_COUNT = 4 };
// Record CUDA events around a launch when profiling is on (no-ops otherwise).
void prof_begin(qdse_ctx* c, int kind);
void prof_end(qdse_ctx* c);

// ---- host grid construction (grid.cpp) -------------------------------------------------------
int gauss_legendre_nodes(int n, double* t, double* v);
void build_instance_grid(const qdse_grid& g, double* sp, double* sq, double* W, double* wt,
                         double* stc, int* sta);
void build_angular(int nt, double* z, double* y, double* s2, double* w);

// ---- kernel launchers (return cudaError_t of the launch) -------------------------------------
cudaError_t launch_precompute(qdse_ctx* c, bool with_omega_derivative);
cudaError_t configure_precompute(int max_nt);
void exp_tables(std::vector<float2>& out);
cudaError_t launch_init_state(qdse_ctx* c, const Ctl& ctl, double* A, double* B, int phase0);
cudaError_t launch_tick(qdse_ctx* c, double* A, double* B);
cudaError_t launch_tick_ring(qdse_ctx* c, double* A, double* B);
cudaError_t launch_tick_narrow(qdse_ctx* c);
cudaError_t launch_tick_slab(qdse_ctx* c, double* A, double* B);
cudaError_t configure_tick_slab();
cudaError_t configure_tick_ring();
cudaError_t tc_setup(qdse_ctx* c);
void tc_free(qdse_ctx* c);
cudaError_t launch_tc_extract(qdse_ctx* c);
cudaError_t launch_tc_sweep(qdse_ctx* c);
cudaError_t launch_group_bands(qdse_ctx* c);
cudaError_t launch_group_params(qdse_ctx* c);
cudaError_t launch_update(qdse_ctx* c, double* A, double* B);
cudaError_t launch_sweep_otf(qdse_ctx* c, const double* A, const double* B, double* FA,
                             double* FB, int only_active);
cudaError_t launch_finish(qdse_ctx* c, double* A, double* B, double* change_out, int* iters,
                          int* status);
cudaError_t launch_residual_fp64(qdse_ctx* c, const double* A, const double* B, double* FA,
                                 double* FB, double* rel, int homogeneous, const float* Khi,
                                 const float* Klo);
cudaError_t launch_jvp(qdse_ctx* c, const double* A, const double* B, const double* vA,
                       const double* vB, double* JA, double* JB);
cudaError_t launch_vjp(qdse_ctx* c, const double* A, const double* B, const double* wA,
                       const double* wB, double* JA, double* JB, int add_g, const double* gA,
                       const double* gB);
cudaError_t launch_condensate(qdse_ctx* c, const double* A, const double* B, double* out);
cudaError_t launch_condensate_vjp(qdse_ctx* c, const double* A, const double* B,
                                  const double* cbar, double* gA, double* gB);
cudaError_t launch_adjoint_update(qdse_ctx* c, double* lam, const double* lam_new, int* n_active);
cudaError_t launch_adjoint_prep(qdse_ctx* c, const double* A, const double* B);
cudaError_t launch_adjoint_mixed_tick(qdse_ctx* c, const double* gA, const double* gB,
                                      int* n_active);
cudaError_t launch_adjoint_sweep(qdse_ctx* c, const double* A, const double* B, const double* gA,
                                 const double* gB);
cudaError_t launch_finish_timeout(qdse_ctx* c, double* A, double* B, double* change_out,
                                  int* iters, int* status);
cudaError_t launch_prep64(qdse_ctx* c, const double* A, const double* B, const double* vA,
                          const double* vB);
cudaError_t launch_rel64(qdse_ctx* c, const double* A, const double* B, const double* FA,
                         const double* FB, double* rel);
cudaError_t launch_adjoint_init(qdse_ctx* c, double* lam, const double* gA, const double* gB,
                                const double* rel, double not_fixed, int phase0);
cudaError_t launch_adjoint_grads(qdse_ctx* c, const double* A, const double* B,
                                 const double* lam, const double* F, const double* Fw,
                                 double* g_params, int* inst_status);

}  // namespace qdse
