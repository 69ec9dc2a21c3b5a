// api.cu -- the C interface of libqdse (declared in include/qdse.h): argument checking, context
// set-up, and the host drivers of the batched successive approximation (Eqs. jifen14-jifen122),
// its mixed-precision refinement and the implicit adjoint.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "qdse_internal.h"

using namespace qdse;

namespace qdse {

static cudaEvent_t next_event(qdse_ctx* c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

void prof_begin(qdse_ctx* c, int kind) {
    if (!c->profiling) return;
    cudaEvent_t a = next_event(c);
    if (!a) return;
    cudaEventRecord(a, c->stream);
    c->prof.push_back({kind, a, nullptr});
}

void prof_end(qdse_ctx* c) {
    if (!c->profiling || c->prof.empty() || c->prof.back().b) return;
    cudaEvent_t b = next_event(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->prof.back().b = b;
}

}  // namespace qdse

namespace {

thread_local std::string g_create_error;

qdse_status fail(qdse_ctx* c, qdse_status st, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return st;
}

qdse_status cuda_fail(qdse_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? QDSE_ERR_OOM : QDSE_ERR_CUDA, m);
}

#define QCHECK(c, expr, where)                                  \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return cuda_fail((c), _e, where); \
    } while (0)

bool finite(double x) { return std::isfinite(x); }

qdse_status check_options(const qdse_options* o, std::string& why) {
    if (!o) { why = "options: null pointer"; return QDSE_ERR_ARG; }
    if (o->precision < QDSE_FP64 || o->precision > QDSE_FP32) { why = "options.precision out of range"; return QDSE_ERR_ARG; }
    if (o->vertex != QDSE_VERTEX_BC && o->vertex != QDSE_VERTEX_RL) { why = "options.vertex out of range"; return QDSE_ERR_ARG; }
    if (!finite(o->cf) || o->cf <= 0) { why = "options.cf must be finite and > 0"; return QDSE_ERR_ARG; }
    if (!finite(o->tol) || o->tol < 0) { why = "options.tol must be finite and >= 0"; return QDSE_ERR_ARG; }
    if (!finite(o->alpha) || o->alpha <= 0 || o->alpha > 1) { why = "options.alpha must be in (0, 1]"; return QDSE_ERR_ARG; }
    if (o->max_iter < 1) { why = "options.max_iter must be >= 1"; return QDSE_ERR_ARG; }
    if (std::isnan(o->time_limit)) { why = "options.time_limit is NaN"; return QDSE_ERR_ARG; }
    if (o->stall_window < 0) { why = "options.stall_window must be >= 0"; return QDSE_ERR_ARG; }
    if (o->stop_cycles != 0 && o->stop_cycles != 1) { why = "options.stop_cycles must be 0 or 1"; return QDSE_ERR_ARG; }
    if (o->shared_kernels != 0 && o->shared_kernels != 1) { why = "options.shared_kernels must be 0 or 1"; return QDSE_ERR_ARG; }
    if (o->shared_kernels) {
        if (o->vertex != QDSE_VERTEX_BC) { why = "options.shared_kernels needs the BC vertex"; return QDSE_ERR_ARG; }
        if (o->precision != QDSE_MIXED && o->precision != QDSE_FP32) { why = "options.shared_kernels needs QDSE_MIXED or QDSE_FP32"; return QDSE_ERR_ARG; }
    }
    return QDSE_OK;
}

qdse_status check_grid(const qdse_grid& g, std::string& why) {
    if (g.n_p < 3 || g.n_p > kMaxN) { why = "grid.n_p must be in [3, 1024]"; return QDSE_ERR_ARG; }
    if (g.n_theta < 1 || g.n_theta > kMaxTheta) { why = "grid.n_theta must be in [1, 512]"; return QDSE_ERR_ARG; }
    if (!finite(g.s_min) || !finite(g.s_max) || g.s_min <= 0 || g.s_max <= g.s_min) {
        why = "grid: need 0 < s_min < s_max, both finite";
        return QDSE_ERR_ARG;
    }
    if (g.grid_mode != QDSE_COLLOCATED && g.grid_mode != QDSE_STAGGERED) { why = "grid.grid_mode out of range"; return QDSE_ERR_ARG; }
    return QDSE_OK;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

void free_ctx(qdse_ctx* c) {
    if (!c) return;
    void* ptrs[] = {c->d_inst, c->d_state, c->d_ctl, c->grid.sp, c->grid.sq, c->grid.W,
                    c->grid.rsp, c->grid.rsq, c->grid.wt, c->grid.stc, c->grid.sta,
                    c->grid.sp32, c->grid.sq32, c->grid.z, c->grid.y, c->grid.s2, c->grid.wz,
                    c->grid.row_inst, c->work.xn64, c->work.r64, c->work.d64, c->work.vec64,
                    c->work.dia64, c->work.x32, c->work.xn32, c->work.vec32, c->work.dia32,
                    c->work.dvec32, c->work.ddia32, c->work.d32, c->work.dvec64, c->work.ddia64,
                    c->work.lam, c->work.lamn, c->d_Khi, c->d_Klo, c->d_Kwhi, c->d_Kwlo,
                    c->d_count, c->d_sweeps, c->d_hostA, c->d_hostI, c->grid.band,
                    c->grid.groups, c->grid.nnz, c->grid.gdesc, c->grid.gphase, c->work.ilist,
                    c->work.glist, c->work.lcount, c->d_tiles, c->d_rel, c->grid.ktd,
                    c->grid.W32, c->grid.wt32, c->grid.stc32, c->grid.expt, c->work.hring, c->work.ticket, c->work.col,
                    c->work.slist, c->grid.slabs, c->work.sphase, c->work.claim,
                    c->work.nlist, c->grid.nfirst};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->h_count) cudaFreeHost(c->h_count);
    if (c->h_inst_pinned) cudaFreeHost(c->h_inst_pinned);
    tc_free(c);
    delete c;
}

// Upload per-instance parameters; reports whether the kernels must be rebuilt.
qdse_status set_params(qdse_ctx* c, const qdse_params* p, bool& rebuild) {
    if (!p) return fail(c, QDSE_ERR_ARG, "params: null pointer");
    rebuild = !(c->opt.reuse_kernels && c->k_valid_for);
    for (int b = 0; b < c->n_inst; ++b) {
        const qdse_params& q = p[b];
        if (!finite(q.D) || q.D < 0 || !finite(q.omega) || q.omega <= 0 || !finite(q.m) ||
            !finite(q.mu)) {
            return fail(c, QDSE_ERR_ARG, "params[" + std::to_string(b) +
                                             "]: need finite D >= 0, omega > 0, m, mu");
        }
        if (q.mu != 0.0)
            return fail(c, QDSE_ERR_UNSUPPORTED, "params[" + std::to_string(b) +
                                                     "]: the vacuum solver needs mu = 0");
        if (c->k_omega[b] != q.omega) rebuild = true;
        if (c->tc && q.omega != p[0].omega)
            return fail(c, QDSE_ERR_ARG, "params[" + std::to_string(b) +
                                             "]: shared kernels need one omega for every instance");
    }
    for (int b = 0; b < c->n_inst; ++b) {
        const HostInst& h = c->hinst[b];
        DevInst& d = c->h_inst_pinned[b];
        d.n = h.g.n_p;
        d.nt = h.g.n_theta;
        d.x_off = h.x_off;
        d.t_off = h.t_off;
        d.k_off = h.k_off;
        d.ld = h.ld;
        d.mode = h.g.grid_mode;
        d.v_off = h.v_off;
        d.g_off = h.g_off;
        d.s_off = h.s_off;
        d.D = p[b].D;
        d.omega = p[b].omega;
        d.m = p[b].m;
    }
    QCHECK(c, cudaMemcpyAsync(c->d_inst, c->h_inst_pinned, sizeof(DevInst) * c->n_inst,
                              cudaMemcpyHostToDevice, c->stream),
           "upload parameters");
    QCHECK(c, launch_group_params(c), "group parameters");
    return QDSE_OK;
}

qdse_status ensure_kernels(qdse_ctx* c, const qdse_params* p, bool rebuild) {
    if (!rebuild) return QDSE_OK;
    QCHECK(c, launch_precompute(c, false), "precompute kernels");
    QCHECK(c, launch_group_bands(c), "group bands");
    if (c->tc) QCHECK(c, launch_tc_extract(c), "tensor-core kernel planes");
    for (int b = 0; b < c->n_inst; ++b) c->k_omega[b] = p[b].omega;
    c->k_valid_for = 1;
    c->kw_valid = 0;
    return QDSE_OK;
}

// The narrow list applies to the ring sweep's separate-update form with the Ball-Chiu vertex
// (the only path whose narrow tiles k_tick_narrow reproduces); the slab, register-only, fused and
// tensor-core paths keep every row group on the group list.
bool narrow_split(const qdse_ctx* c) {
    return c->narrow_ok && c->sweep_kind == 1 && !c->fused_update && !c->tc &&
           c->opt.vertex == QDSE_VERTEX_BC &&
           (c->opt.precision == QDSE_MIXED || c->opt.precision == QDSE_FP32);
}

Ctl make_ctl(const qdse_ctx* c) {
    Ctl t{};
    t.kappa = c->opt.cf / (8.0 * kPi * kPi * kPi);
    t.tol = c->opt.tol;
    t.sw_tol = std::fmax(1e-5, c->opt.tol);
    t.inner_tol = 1e-3;
    t.alpha = c->opt.alpha;
    t.max_iter = c->opt.max_iter;
    t.max_inner = 400;
    t.max_fp32 = c->opt.max_iter;
    t.vertex = c->opt.vertex;
    t.precision = c->opt.precision;
    t.final_phase = (c->opt.precision == QDSE_FP32) ? PH_PICARD32 : PH_PICARD64;
    t.never_converge = 0;
    t.stall_copies = c->stall_copies;
    t.stall_window = c->opt.stall_window;
    t.stop_cycles = c->opt.stop_cycles;
    t.tc_picard = c->tc;
    t.slab_lists = c->sweep_kind == 2;
    t.narrow_split = narrow_split(c) ? 1 : 0;
    return t;
}

void reset_stats(qdse_ctx* c) {
    c->launches = 0;
    c->sweeps32 = 0;
    c->sweeps64 = 0;
    c->polls = 0;
    c->ev_used = 0;
    c->prof.clear();
    if (c->d_sweeps) cudaMemsetAsync(c->d_sweeps, 0, 4 * sizeof(unsigned long long), c->stream);
}

// One tick: the sweep for the path in use and, where the sweep does not update instances itself,
// the per-instance update.  `last` zeroes the poll counter first (it counts the instances still
// running after this tick).
cudaError_t launch_one_tick(qdse_ctx* c, double* A, double* B, bool last) {
    const bool otf = (c->opt.precision == QDSE_FP64);
    cudaError_t e = cudaSuccess;
    if (last) e = cudaMemsetAsync(c->d_count, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    if (!otf && c->tc) {
        // FP32 Picard rows of the whole batch on the tensor cores; the sweep below takes the
        // row groups of every other phase
        e = launch_tc_sweep(c);
        if (e != cudaSuccess) return e;
    }
    if (otf) {
        e = launch_sweep_otf(c, A, B, c->work.xn64, c->work.xn64 + c->n_total, 1);
    } else if (c->sweep_kind == 2) {
        e = launch_tick_slab(c, A, B);
    } else if (c->sweep_kind == 1) {
        // the ring sweep advances every instance itself once its last row group is swept
        e = launch_tick_ring(c, A, B);
        if (e != cudaSuccess || c->fused_update) return e;
        if (narrow_split(c)) e = launch_tick_narrow(c);
    } else {
        e = launch_tick(c, A, B);
    }
    if (e != cudaSuccess) return e;
    return launch_update(c, A, B);
}

constexpr int kGraphTicks = 48;  // ticks per captured chunk: a multiple of 3 keeps the
                                 // active-list buffers (mod 3) in step

// Capture kGraphTicks ticks on the internal stream into c->gexec (A, B fixed).
qdse_status capture_chunk(qdse_ctx* c, double* A, double* B, int path) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    const long long tick0 = c->tick, launches0 = c->launches;
    QCHECK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < kGraphTicks && e == cudaSuccess; ++t)
        e = launch_one_tick(c, A, B, t == kGraphTicks - 1);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    c->tick = tick0;
    c->g_launches = c->launches - launches0;
    c->launches = launches0;
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(c, e, "capture a chunk of ticks");
    }
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, e, "instantiate the tick graph");
    }
    c->g_A = A;
    c->g_B = B;
    c->g_path = path;
    return QDSE_OK;
}

// The batched successive approximation: ticks of (sweep rows, update instances) with the number
// of unfinished instances polled between chunks.  n_ticks < 0 means "until every instance has
// finished"; otherwise exactly n_ticks ticks without polling.  Solves run on an internal stream
// (ordered after and before the caller's stream by events) in replayed CUDA graphs of
// kGraphTicks ticks, unless per-launch profiling is on.
qdse_status run_ticks(qdse_ctx* c, double* A, double* B, long long n_ticks, bool& timed_out) {
    timed_out = false;
    QCHECK(c, cudaMemsetAsync(c->d_count, 0, 2 * sizeof(int), c->stream), "reset flags");
    const auto t0 = std::chrono::steady_clock::now();
    if (n_ticks >= 0) {
        for (long long t = 0; t < n_ticks; ++t) QCHECK(c, launch_one_tick(c, A, B, false), "tick");
        return QDSE_OK;
    }
    const bool graphs = !c->profiling;
    cudaStream_t user = c->stream;
    if (graphs) {
        QCHECK(c, cudaEventRecord(c->ev_in, user), "order the solve stream");
        QCHECK(c, cudaStreamWaitEvent(c->gstream, c->ev_in, 0), "order the solve stream");
        c->stream = c->gstream;
    }
    const int path = (c->opt.precision == QDSE_FP64)
                         ? -2
                         : 4 * c->sweep_kind + c->ring_shape + (narrow_split(c) ? 16 : 0);
    int chunk = 4;
    qdse_status st = QDSE_OK;
    while (true) {
        if (graphs) {
            if (!c->gexec || c->g_A != A || c->g_B != B || c->g_path != path) {
                st = capture_chunk(c, A, B, path);
                if (st != QDSE_OK) break;
            }
            cudaError_t e = cudaGraphLaunch(c->gexec, c->stream);
            if (e != cudaSuccess) {
                st = cuda_fail(c, e, "launch the tick graph");
                break;
            }
            c->tick += kGraphTicks;
            c->launches += c->g_launches;
        } else {
            cudaError_t e = cudaSuccess;
            for (int t = 0; t < chunk && e == cudaSuccess; ++t)
                e = launch_one_tick(c, A, B, t == chunk - 1);
            if (e != cudaSuccess) {
                st = cuda_fail(c, e, "tick");
                break;
            }
            if (chunk < 64) chunk *= 2;
        }
        cudaError_t e = cudaMemcpyAsync(c->h_count, c->d_count, 2 * sizeof(int),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "poll");
            break;
        }
        c->polls++;
        if (c->h_count[1] != 0) {
            timed_out = true;
            st = fail(c, QDSE_ERR_TIMEOUT, "a bounded device wait ran out in the sweep kernel");
            break;
        }
        if (*c->h_count == 0) break;
        if (c->opt.time_limit > 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > c->opt.time_limit) {
                timed_out = true;
                break;
            }
        }
    }
    if (graphs) {
        c->stream = user;
        cudaError_t e = cudaEventRecord(c->ev_out, c->gstream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user, c->ev_out, 0);
        if (e != cudaSuccess && st == QDSE_OK) st = cuda_fail(c, e, "order the caller's stream");
    }
    return st;
}

qdse_status check_ptr(qdse_ctx* c, const void* p, const char* name) {
    if (!p) return fail(c, QDSE_ERR_ARG, std::string(name) + ": null pointer");
    return QDSE_OK;
}

qdse_status create_impl(const qdse_grid* g, int n_inst, bool ragged, const qdse_options* o,
                        qdse_ctx** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, QDSE_ERR_ARG, "out: null pointer");
    *out = nullptr;
    if (!g) return fail(nullptr, QDSE_ERR_ARG, "grid: null pointer");
    if (n_inst < 1) return fail(nullptr, QDSE_ERR_ARG, "n_inst must be >= 1");
    std::string why;
    if (check_options(o, why) != QDSE_OK) return fail(nullptr, QDSE_ERR_ARG, why);
    for (int b = 0; b < (ragged ? n_inst : 1); ++b)
        if (check_grid(g[b], why) != QDSE_OK)
            return fail(nullptr, QDSE_ERR_ARG, "instance " + std::to_string(b) + ": " + why);
    if (o->shared_kernels && (ragged || g[0].grid_mode != QDSE_COLLOCATED))
        return fail(nullptr, QDSE_ERR_ARG,
                    "options.shared_kernels needs one COLLOCATED grid for every instance "
                    "(qdse_create)");

    qdse_ctx* c = new (std::nothrow) qdse_ctx();
    if (!c) return fail(nullptr, QDSE_ERR_OOM, "host allocation");
    c->opt = *o;
    c->stream = (cudaStream_t)o->stream;
    c->n_inst = n_inst;
    c->hinst.resize(n_inst);
    c->k_omega.assign(n_inst, NAN);
    std::map<int, int> t_of;  // angular node count -> offset of its shared table
    long long k = 0;
    int x = 0, t = 0, v = 0, ng = 0;
    for (int b = 0; b < n_inst; ++b) {
        HostInst& h = c->hinst[b];
        h.g = ragged ? g[b] : g[0];
        h.x_off = x;
        h.ld = (h.g.n_p + 3) & ~3;
        h.v_off = v;
        // shared kernels: every instance reads the one kernel block of instance 0
        h.k_off = o->shared_kernels ? 0 : k;
        x += h.g.n_p;
        v += h.ld;
        ng += (h.g.n_p + kRows - 1) / kRows;
        if (!o->shared_kernels || b == 0) k += 3LL * h.g.n_p * h.ld;
        if (!t_of.count(h.g.n_theta)) {
            t_of[h.g.n_theta] = t;
            t += h.g.n_theta;
        }
        h.t_off = t_of[h.g.n_theta];
        if (h.g.n_p > c->max_n) c->max_n = h.g.n_p;
        if (h.ld > c->ld_max) c->ld_max = h.ld;
        if (h.g.n_theta > c->max_nt) c->max_nt = h.g.n_theta;
        if (h.g.grid_mode == QDSE_STAGGERED) c->any_staggered = true;
    }
    c->n_total = x;
    c->nv_total = v;
    c->n_groups = ng;
    c->t_total = t;
    c->k_total = k;

    // host grids
    const int N = c->n_total;
    std::vector<double> sp(N), sq(N), W(N), wt(N), stc(3 * (size_t)N), rsp(N), rsq(N);
    std::vector<int> sta(N), row_inst(N);
    // precompute tiles: collocated grids only the upper triangle (J >= I), staggered all
    std::vector<int4> tiles;
    for (int b = 0; b < (o->shared_kernels ? 1 : n_inst); ++b) {
        const HostInst& h = c->hinst[b];
        const int T = (h.g.n_p + kTile - 1) / kTile;
        for (int I = 0; I < T; ++I)
            for (int J = (h.g.grid_mode == QDSE_COLLOCATED ? I : 0); J < T; ++J)
                tiles.push_back(make_int4(b, I, J, 0));
    }
    c->n_tiles = (int)tiles.size();
    std::vector<int2> groups;
    std::vector<GroupDesc> gdesc;
    std::vector<SlabRec> slabs;
    groups.reserve(ng);
    gdesc.reserve(ng);
    for (int b = 0; b < n_inst; ++b) {
        HostInst& h = c->hinst[b];
        h.g_off = (int)groups.size();
        h.s_off = (int)slabs.size();
        const int ngb = (h.g.n_p + kRows - 1) / kRows;
        for (int g0 = 0; g0 < ngb; g0 += kSlabGroups) {
            SlabRec r{};
            r.b = b;
            r.g0 = g0;
            r.ng = std::min(kSlabGroups, ngb - g0);
            r.x_off = h.x_off;
            r.v_off = h.v_off;
            r.n = h.g.n_p;
            r.ld = h.ld;
            r.mode = h.g.grid_mode;
            r.k_off = h.k_off;
            for (int q = 0; q < kSlabGroups; ++q) r.band[q] = make_int2(0, q < r.ng ? h.ld : 0);
            slabs.push_back(r);
        }
        for (int i0 = 0; i0 < h.g.n_p; i0 += kRows) {
            groups.push_back(make_int2(b, i0));
            GroupDesc d{};
            d.b = b;
            d.i0 = i0;
            d.nr = std::min(kRows, h.g.n_p - i0);
            d.jlo = 0;
            d.jhi = h.ld;  // narrowed to the band union after every kernel precompute
            d.v_off = h.v_off;
            d.x_off = h.x_off;
            d.ld = h.ld;
            d.kbase = h.k_off + (long long)i0 * 3 * h.ld;
            d.mode = h.g.grid_mode;
            d.ng = (h.g.n_p + kRows - 1) / kRows;
            gdesc.push_back(d);
        }
    }
    std::vector<float> sp32(N), sq32(N), W32(N), wt32(N), stc32(3 * (size_t)N);
    for (int b = 0; b < n_inst; ++b) {
        const HostInst& h = c->hinst[b];
        const int o0 = h.x_off;
        build_instance_grid(h.g, &sp[o0], &sq[o0], &W[o0], &wt[o0], &stc[3 * (size_t)o0],
                            &sta[o0]);
        for (int j = 0; j < h.g.n_p; ++j) row_inst[o0 + j] = b;
    }
    for (int j = 0; j < N; ++j) {
        rsp[j] = std::sqrt(sp[j]);
        rsq[j] = std::sqrt(sq[j]);
        sp32[j] = (float)sp[j];
        sq32[j] = (float)sq[j];
        W32[j] = (float)W[j];
        wt32[j] = (float)wt[j];
        for (int k = 0; k < 3; ++k) stc32[3 * (size_t)j + k] = (float)stc[3 * (size_t)j + k];
    }
    std::vector<double> z(t), y(t), s2(t), wz(t);
    for (auto& kv : t_of) build_angular(kv.first, &z[kv.second], &y[kv.second], &s2[kv.second], &wz[kv.second]);
    c->h_sp = sp;
    c->h_sq = sq;
    c->h_W = W;

#define CALLOC(ptr, n)                                                      \
    do {                                                                    \
        cudaError_t _e = dalloc(&(ptr), (n));                               \
        if (_e != cudaSuccess) {                                            \
            qdse_status _s = cuda_fail(nullptr, _e, "allocate " #ptr);      \
            free_ctx(c);                                                    \
            return _s;                                                      \
        }                                                                   \
    } while (0)
    CALLOC(c->d_inst, n_inst);
    CALLOC(c->d_state, n_inst);
    CALLOC(c->d_ctl, 1);
    CALLOC(c->grid.sp, N);
    CALLOC(c->grid.sq, N);
    CALLOC(c->grid.W, N);
    CALLOC(c->grid.rsp, N);
    CALLOC(c->grid.rsq, N);
    CALLOC(c->grid.wt, N);
    CALLOC(c->grid.stc, 3 * (size_t)N);
    CALLOC(c->grid.sta, N);
    CALLOC(c->grid.sp32, N);
    CALLOC(c->grid.ktd, N);
    CALLOC(c->grid.W32, N);
    CALLOC(c->grid.wt32, N);
    CALLOC(c->grid.stc32, 3 * (size_t)N);
    CALLOC(c->grid.sq32, N);
    CALLOC(c->grid.z, t);
    CALLOC(c->grid.y, t);
    CALLOC(c->grid.s2, t);
    CALLOC(c->grid.wz, t);
    CALLOC(c->grid.row_inst, N);
    CALLOC(c->grid.band, N);
    CALLOC(c->grid.nnz, n_inst);
    CALLOC(c->grid.nfirst, n_inst);
    std::vector<float2> expt;
    exp_tables(expt);
    CALLOC(c->grid.expt, expt.size());
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    CALLOC(c->work.ilist, 3 * (size_t)n_inst);
    CALLOC(c->work.glist, 3 * (size_t)ng);
    CALLOC(c->work.nlist, 3 * (size_t)ng);
    CALLOC(c->work.lcount, 12);
    c->n_slabs = (int)slabs.size();
    c->work.n_slabs = c->n_slabs;
    CALLOC(c->work.slist, 3 * (size_t)c->n_slabs);
    CALLOC(c->work.sphase, c->n_slabs);
    CALLOC(c->work.claim, 3);
    CALLOC(c->grid.slabs, c->n_slabs);
    CALLOC(c->work.hring, (size_t)kHashRing * n_inst);
    CALLOC(c->work.ticket, n_inst);
    CALLOC(c->work.col, 2 * (size_t)N);
    c->work.n_inst = n_inst;
    c->work.n_groups = ng;
    CALLOC(c->grid.groups, ng);
    CALLOC(c->grid.gdesc, ng);
    CALLOC(c->d_tiles, c->n_tiles);
    CALLOC(c->d_rel, n_inst);
    CALLOC(c->grid.gphase, ng);
    CALLOC(c->work.xn64, 2 * (size_t)N);
    CALLOC(c->work.r64, 2 * (size_t)N);
    CALLOC(c->work.d64, 2 * (size_t)N);
    CALLOC(c->work.vec64, 5 * (size_t)N);
    CALLOC(c->work.dia64, 2 * (size_t)N);
    CALLOC(c->work.x32, 2 * (size_t)N);
    CALLOC(c->work.xn32, 2 * (size_t)N);
    CALLOC(c->work.vec32, 5 * (size_t)v);
    CALLOC(c->work.dia32, 2 * (size_t)N);
    CALLOC(c->work.dvec32, 5 * (size_t)v);
    CALLOC(c->work.ddia32, 2 * (size_t)N);
    CALLOC(c->work.d32, 2 * (size_t)N);
    CALLOC(c->work.dvec64, 5 * (size_t)N);
    CALLOC(c->work.ddia64, 2 * (size_t)N);
    CALLOC(c->work.lam, 2 * (size_t)N);
    CALLOC(c->work.lamn, 2 * (size_t)N);
    CALLOC(c->d_Khi, (size_t)k);
    CALLOC(c->d_Klo, (size_t)k);
    CALLOC(c->d_count, 2);
    CALLOC(c->d_sweeps, 4);
    CALLOC(c->d_hostA, 2 * (size_t)N);
    CALLOC(c->d_hostI, 2 * (size_t)n_inst);
#undef CALLOC
    c->d_err = c->d_count + 1;
    cudaError_t e = cudaMallocHost((void**)&c->h_count, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_inst_pinned, sizeof(DevInst) * n_inst);
    if (e != cudaSuccess) {
        qdse_status s = cuda_fail(nullptr, e, "pinned host allocation");
        free_ctx(c);
        return s;
    }
    struct Up { void* d; const void* h; size_t bytes; } ups[] = {
        {c->grid.sp, sp.data(), sizeof(double) * N}, {c->grid.sq, sq.data(), sizeof(double) * N},
        {c->grid.W, W.data(), sizeof(double) * N}, {c->grid.rsp, rsp.data(), sizeof(double) * N},
        {c->grid.rsq, rsq.data(), sizeof(double) * N}, {c->grid.wt, wt.data(), sizeof(double) * N},
        {c->grid.stc, stc.data(), sizeof(double) * 3 * (size_t)N},
        {c->grid.sta, sta.data(), sizeof(int) * N}, {c->grid.sp32, sp32.data(), sizeof(float) * N},
        {c->grid.sq32, sq32.data(), sizeof(float) * N}, {c->grid.W32, W32.data(), sizeof(float) * N},
        {c->grid.wt32, wt32.data(), sizeof(float) * N},
        {c->grid.stc32, stc32.data(), sizeof(float) * 3 * (size_t)N},
        {c->grid.z, z.data(), sizeof(double) * t},
        {c->grid.y, y.data(), sizeof(double) * t}, {c->grid.s2, s2.data(), sizeof(double) * t},
        {c->grid.wz, wz.data(), sizeof(double) * t},
        {c->grid.row_inst, row_inst.data(), sizeof(int) * N},
        {c->grid.groups, groups.data(), sizeof(int2) * ng},
        {c->grid.gdesc, gdesc.data(), sizeof(GroupDesc) * ng},
        {c->d_tiles, tiles.data(), sizeof(int4) * c->n_tiles},
        {c->grid.expt, expt.data(), sizeof(float2) * expt.size()},
        {c->grid.slabs, slabs.data(), sizeof(SlabRec) * slabs.size()}};
    for (auto& u : ups) {
        e = cudaMemcpy(u.d, u.h, u.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            qdse_status s = cuda_fail(nullptr, e, "upload grid");
            free_ctx(c);
            return s;
        }
    }
    c->work.nv = v;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        qdse_status s = cuda_fail(nullptr, e, "create the solve stream");
        free_ctx(c);
        return s;
    }
    e = configure_precompute(c->max_nt);
    if (e != cudaSuccess) {
        qdse_status s = cuda_fail(nullptr, e, "configure the precompute kernel");
        free_ctx(c);
        return s;
    }
    {
        // FP32 sweep kernel: the shared-memory ring by default; QDSE_SWEEP=groups selects the
        // register-only row-group kernel (same results up to rounding order)
        const char* k = std::getenv("QDSE_SWEEP");
        const bool ring_ok = configure_tick_ring() == cudaSuccess;
        cudaGetLastError();
        const bool slab_ok = configure_tick_slab() == cudaSuccess;
        c->slab_ok = slab_ok ? 1 : 0;
        cudaGetLastError();
        c->sweep_kind = ring_ok ? 1 : 0;
        if (k && std::string(k) == "slab" && slab_ok) c->sweep_kind = 2;
        if (k && std::string(k) == "groups") c->sweep_kind = 0;
        // QDSE_FUSED_UPDATE=1: the ring sweep advances each instance itself (one launch per tick;
        // the same arithmetic in the same order as the separate update launch, but measured
        // slower: the update's dependent loads by one warp, among the sweep's 12 warps per SM)
        // QDSE_RING=8x3 / 6x4: fewer warps per block, each with more tile slots in flight and its
        // copying side further ahead (the default is 12 warps x 2 slots)
        const char* rs = std::getenv("QDSE_RING");
        c->ring_shape = (rs && std::string(rs) == "8x3") ? 1 : (rs && std::string(rs) == "6x4") ? 2 : 0;
        const char* fu = std::getenv("QDSE_FUSED_UPDATE");
        c->fused_update = (fu && std::string(fu) == "1") ? 1 : 0;
        // QDSE_NARROW=0: the ring sweep takes the narrow row groups too (bitwise the same results)
        const char* nw = std::getenv("QDSE_NARROW");
        c->narrow_ok = (nw && std::string(nw) == "0") ? 0 : 1;
        // kernel matrices: double-float on the FP32 pipe by default; QDSE_PRECOMPUTE=fp64
        // selects the FP64 kernel (the same entries to about 1e-14)
        const char* pk = std::getenv("QDSE_PRECOMPUTE");
        c->precompute_kind = (pk && std::string(pk) == "fp64") ? 0 : 1;
        // test of the sweep's bounded waits (tests only): every tile wait runs out
        const char* st = std::getenv("QDSE_TEST_STALL");
        c->stall_copies = (st && std::string(st) == "1") ? 1 : 0;
    }
    if (o->shared_kernels) {
        // one grid for every instance (checked above), collocated
        c->tc = 1;
        c->tc_n = c->hinst[0].g.n_p;
        c->fused_update = 0;  // the update launch advances the instances the product swept
        e = tc_setup(c);
        if (e != cudaSuccess) {
            qdse_status s = cuda_fail(nullptr, e, "set up the tensor-core sweep");
            free_ctx(c);
            return s;
        }
    }
    // zero the padding of the node vectors once; descriptors get their layout now and their
    // parameters on every call
    e = cudaMemset(c->work.vec32, 0, sizeof(float) * 5 * (size_t)v);
    if (e == cudaSuccess) e = cudaMemset(c->work.dvec32, 0, sizeof(float) * 5 * (size_t)v);
    if (e == cudaSuccess) e = cudaMemset(c->grid.ktd, 0, sizeof(float) * (size_t)c->n_total);
    if (e == cudaSuccess) {
        std::vector<qdse_params> zero(n_inst, qdse_params{0.0, 1.0, 0.0, 0.0});
        bool rb = false;
        c->stream = nullptr;
        if (set_params(c, zero.data(), rb) != QDSE_OK) e = cudaErrorUnknown;
        else e = cudaStreamSynchronize(nullptr);
        c->stream = (cudaStream_t)o->stream;
        for (int b = 0; b < n_inst; ++b) c->k_omega[b] = NAN;
    }
    if (e != cudaSuccess) {
        qdse_status s = cuda_fail(nullptr, e, "initialise workspaces");
        free_ctx(c);
        return s;
    }
    *out = c;
    return QDSE_OK;
}

}  // namespace

extern "C" {

qdse_options qdse_default_options(void) {
    qdse_options o;
    o.precision = QDSE_MIXED;
    o.vertex = QDSE_VERTEX_BC;
    o.cf = 4.0 / 3.0;
    o.tol = 1e-10;
    o.alpha = 1.0;
    o.max_iter = 20000;
    o.time_limit = 0.0;
    o.reuse_kernels = 0;
    o.stall_window = 0;
    o.stop_cycles = 1;
    o.shared_kernels = 0;
    o.stream = nullptr;
    return o;
}

qdse_status qdse_create(const qdse_grid* g, int n_inst, const qdse_options* o, qdse_ctx** out) {
    try {
        return create_impl(g, n_inst, false, o, out);
    } catch (...) {
        return fail(nullptr, QDSE_ERR_OOM, "host exception during create");
    }
}

qdse_status qdse_create_ragged(const qdse_grid* g, int n_inst, const qdse_options* o,
                               qdse_ctx** out) {
    try {
        return create_impl(g, n_inst, true, o, out);
    } catch (...) {
        return fail(nullptr, QDSE_ERR_OOM, "host exception during create");
    }
}

void qdse_destroy(qdse_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

const char* qdse_last_error(const qdse_ctx* c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

qdse_status qdse_sizes(const qdse_ctx* c, int* n_inst, int* n_total) {
    if (!c) return QDSE_ERR_ARG;
    if (n_inst) *n_inst = c->n_inst;
    if (n_total) *n_total = c->n_total;
    return QDSE_OK;
}

qdse_status qdse_layout(const qdse_ctx* c, int* x_off) {
    if (!c || !x_off) return QDSE_ERR_ARG;
    for (int b = 0; b < c->n_inst; ++b) x_off[b] = c->hinst[b].x_off;
    x_off[c->n_inst] = c->n_total;
    return QDSE_OK;
}

qdse_status qdse_grid_nodes(const qdse_ctx* c, double* s_p, double* s_q, double* W) {
    if (!c) return QDSE_ERR_ARG;
    const size_t bytes = sizeof(double) * c->n_total;
    if (s_p) std::memcpy(s_p, c->h_sp.data(), bytes);
    if (s_q) std::memcpy(s_q, c->h_sq.data(), bytes);
    if (W) std::memcpy(W, c->h_W.data(), bytes);
    return QDSE_OK;
}

qdse_status qdse_set_options(qdse_ctx* c, const qdse_options* o) {
    if (!c) return QDSE_ERR_ARG;
    std::string why;
    if (check_options(o, why) != QDSE_OK) return fail(c, QDSE_ERR_ARG, why);
    c->opt = *o;
    c->stream = (cudaStream_t)o->stream;
    return QDSE_OK;
}

qdse_status qdse_autotune(qdse_ctx* c, const qdse_params* p, const double* A0, const double* B0,
                          int max_sweeps, int* choice, double* ms) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    if (max_sweeps < 0) return fail(c, QDSE_ERR_ARG, "max_sweeps must be >= 0");
    if (check_ptr(c, A0, "A") || check_ptr(c, B0, "B")) return QDSE_ERR_ARG;
    struct Cand {
        int kind, shape;
    };
    const Cand cands[kTuneCandidates] = {{1, 0}, {1, 1}, {1, 2}, {2, 0}, {0, 0}};
    int current = 0;
    for (int k = 0; k < kTuneCandidates; ++k)
        if (cands[k].kind == c->sweep_kind && cands[k].shape == c->ring_shape) current = k;
    if (ms)
        for (int k = 0; k < kTuneCandidates; ++k) ms[k] = -1.0;
    // FP64-only contexts and the tensor-core sweep have no per-instance FP32 sweep to choose
    if (c->opt.precision == QDSE_FP64 || c->tc || c->fused_update) {
        if (choice) *choice = current;
        return QDSE_OK;
    }
    reset_stats(c);
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    s = ensure_kernels(c, p, rebuild);
    if (s != QDSE_OK) return s;
    const size_t bytes = sizeof(double) * (size_t)c->n_total;
    double *A = nullptr, *B = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&A, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B, bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int kind0 = c->sweep_kind, shape0 = c->ring_shape;
    int best = current;
    float best_ms = 0.f;
    bool timed = false;
    s = QDSE_OK;
    for (int k = 0; k < kTuneCandidates && e == cudaSuccess && s == QDSE_OK; ++k) {
        if (cands[k].kind == 2 && !c->slab_ok) continue;
        c->sweep_kind = cands[k].kind;
        c->ring_shape = cands[k].shape;
        // one solve of the batch, as qdse_solve runs it (capped at max_sweeps when > 0)
        Ctl ctl = make_ctl(c);
        if (max_sweeps > 0) ctl.max_iter = std::min(ctl.max_iter, max_sweeps);
        const int phase0 = (c->opt.precision == QDSE_MIXED || c->opt.precision == QDSE_FP32)
                               ? PH_PICARD32
                               : PH_PICARD64;
        e = cudaMemcpyAsync(A, A0, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B, B0, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = launch_init_state(c, ctl, A, B, phase0);
        if (e != cudaSuccess) break;
        bool to = false;
        s = run_ticks(c, A, B, -1, to);
        if (s != QDSE_OK || to) {
            if (s == QDSE_OK) s = fail(c, QDSE_ERR_TIMEOUT, "time limit reached while tuning");
            break;
        }
        e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) break;
        if (ms) ms[k] = t;
        if (!timed || t < best_ms) {
            best = k;
            best_ms = t;
            timed = true;
        }
    }
    if (A) cudaFree(A);
    if (B) cudaFree(B);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->sweep_kind = kind0;
    c->ring_shape = shape0;
    if (c->gexec) {  // the captured ticks hold the trial's arrays and kernel
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (s != QDSE_OK) return s;
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    c->sweep_kind = cands[best].kind;
    c->ring_shape = cands[best].shape;
    if (choice) *choice = best;
    return QDSE_OK;
}

qdse_status qdse_iterate(qdse_ctx* c, const qdse_params* p, double* A, double* B, int n_sweeps,
                         double* max_rel_change) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    reset_stats(c);
    if (n_sweeps < 0) return fail(c, QDSE_ERR_ARG, "n_sweeps must be >= 0");
    if (check_ptr(c, A, "A") || check_ptr(c, B, "B")) return QDSE_ERR_ARG;
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    if (n_sweeps == 0) return QDSE_OK;
    if (c->opt.precision != QDSE_FP64) {
        s = ensure_kernels(c, p, rebuild);
        if (s != QDSE_OK) return s;
    }
    Ctl ctl = make_ctl(c);
    ctl.never_converge = 1;
    ctl.max_iter = n_sweeps;
    ctl.final_phase = (c->opt.precision == QDSE_MIXED || c->opt.precision == QDSE_FP32) ? PH_PICARD32 : PH_PICARD64;
    const int phase0 = ctl.final_phase;
    QCHECK(c, launch_init_state(c, ctl, A, B, phase0), "init");
    bool to = false;
    s = run_ticks(c, A, B, n_sweeps, to);
    if (s != QDSE_OK) return s;
    QCHECK(c, launch_finish(c, A, B, max_rel_change, nullptr, nullptr), "finish");
    return QDSE_OK;
}

qdse_status qdse_solve(qdse_ctx* c, const qdse_params* p, double* A, double* B, int* iters,
                       int* inst_status) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    reset_stats(c);
    if (check_ptr(c, A, "A") || check_ptr(c, B, "B")) return QDSE_ERR_ARG;
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    if (c->opt.precision != QDSE_FP64) {
        s = ensure_kernels(c, p, rebuild);
        if (s != QDSE_OK) return s;
    }
    Ctl ctl = make_ctl(c);
    const int phase0 = (c->opt.precision == QDSE_MIXED || c->opt.precision == QDSE_FP32) ? PH_PICARD32 : PH_PICARD64;
    QCHECK(c, launch_init_state(c, ctl, A, B, phase0), "init");
    bool timed_out = false;
    s = run_ticks(c, A, B, -1, timed_out);
    if (s != QDSE_OK && !timed_out) return s;
    if (timed_out) {
        // a bounded device wait ran out (s) or the host time limit was reached
        const std::string why = (s == QDSE_ERR_TIMEOUT)
                                    ? c->err
                                    : std::string("time limit reached before every instance finished");
        QCHECK(c, launch_finish_timeout(c, A, B, nullptr, iters, inst_status), "finish");
        QCHECK(c, cudaStreamSynchronize(c->stream), "sync");
        return fail(c, QDSE_ERR_TIMEOUT, why);
    }
    QCHECK(c, launch_finish(c, A, B, nullptr, iters, inst_status), "finish");
    QCHECK(c, cudaStreamSynchronize(c->stream), "sync");
    return QDSE_OK;
}

qdse_status qdse_solve_host(qdse_ctx* c, const qdse_params* p, double* A, double* B, int* iters,
                            int* inst_status) {
    if (!c) return QDSE_ERR_ARG;
    if (check_ptr(c, A, "A") || check_ptr(c, B, "B")) return QDSE_ERR_ARG;
    const size_t bytes = sizeof(double) * c->n_total;
    double* dA = c->d_hostA;
    double* dB = c->d_hostA + c->n_total;
    QCHECK(c, cudaMemcpyAsync(dA, A, bytes, cudaMemcpyHostToDevice, c->stream), "copy A in");
    QCHECK(c, cudaMemcpyAsync(dB, B, bytes, cudaMemcpyHostToDevice, c->stream), "copy B in");
    qdse_status s = qdse_solve(c, p, dA, dB, c->d_hostI, c->d_hostI + c->n_inst);
    if (s != QDSE_OK && s != QDSE_ERR_TIMEOUT) return s;
    QCHECK(c, cudaMemcpyAsync(A, dA, bytes, cudaMemcpyDeviceToHost, c->stream), "copy A out");
    QCHECK(c, cudaMemcpyAsync(B, dB, bytes, cudaMemcpyDeviceToHost, c->stream), "copy B out");
    if (iters)
        QCHECK(c, cudaMemcpyAsync(iters, c->d_hostI, sizeof(int) * c->n_inst,
                                  cudaMemcpyDeviceToHost, c->stream), "copy iters");
    if (inst_status)
        QCHECK(c, cudaMemcpyAsync(inst_status, c->d_hostI + c->n_inst, sizeof(int) * c->n_inst,
                                  cudaMemcpyDeviceToHost, c->stream), "copy status");
    QCHECK(c, cudaStreamSynchronize(c->stream), "sync");
    return s;
}

qdse_status qdse_residual(qdse_ctx* c, const qdse_params* p, const double* A, const double* B,
                          double* FA, double* FB, double* rel_res) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    reset_stats(c);
    if (check_ptr(c, A, "A") || check_ptr(c, B, "B")) return QDSE_ERR_ARG;
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    Ctl ctl = make_ctl(c);
    QCHECK(c, cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream), "ctl");
    double* oA = FA ? FA : c->work.xn64;
    double* oB = FB ? FB : c->work.xn64 + c->n_total;
    if (c->opt.precision == QDSE_FP64) {
        QCHECK(c, launch_prep64(c, A, B, nullptr, nullptr), "prep");
        QCHECK(c, launch_sweep_otf(c, A, B, oA, oB, 0), "fp64 sweep");
        if (rel_res) QCHECK(c, launch_rel64(c, A, B, oA, oB, rel_res), "rel");
    } else {
        s = ensure_kernels(c, p, rebuild);
        if (s != QDSE_OK) return s;
        QCHECK(c, launch_residual_fp64(c, A, B, oA, oB, rel_res, 0, c->d_Khi, c->d_Klo), "residual");
    }
    return QDSE_OK;
}

qdse_status qdse_jvp(qdse_ctx* c, const qdse_params* p, const double* A, const double* B,
                     const double* vA, const double* vB, double* JvA, double* JvB) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    reset_stats(c);
    const void* ptrs[] = {A, B, vA, vB, JvA, JvB};
    for (const void* q : ptrs)
        if (!q) return fail(c, QDSE_ERR_ARG, "jvp: null pointer");
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    s = ensure_kernels(c, p, rebuild);
    if (s != QDSE_OK) return s;
    Ctl ctl = make_ctl(c);
    QCHECK(c, cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream), "ctl");
    QCHECK(c, launch_jvp(c, A, B, vA, vB, JvA, JvB), "jvp");
    return QDSE_OK;
}

qdse_status qdse_vjp(qdse_ctx* c, const qdse_params* p, const double* A, const double* B,
                     const double* wA, const double* wB, double* JtA, double* JtB) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    reset_stats(c);
    const void* ptrs[] = {A, B, wA, wB, JtA, JtB};
    for (const void* q : ptrs)
        if (!q) return fail(c, QDSE_ERR_ARG, "vjp: null pointer");
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    s = ensure_kernels(c, p, rebuild);
    if (s != QDSE_OK) return s;
    Ctl ctl = make_ctl(c);
    QCHECK(c, cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream), "ctl");
    QCHECK(c, launch_vjp(c, A, B, wA, wB, JtA, JtB, 0, nullptr, nullptr), "vjp");
    return QDSE_OK;
}

qdse_status qdse_adjoint(qdse_ctx* c, const qdse_params* p, const double* A, const double* B,
                         const double* gA, const double* gB, double* g_params,
                         double* lambda_out, int* inst_status) {
    if (!c) return QDSE_ERR_ARG;
    c->err.clear();
    reset_stats(c);
    const void* ptrs[] = {A, B, gA, gB, g_params};
    for (const void* q : ptrs)
        if (!q) return fail(c, QDSE_ERR_ARG, "adjoint: null pointer");
    bool rebuild = false;
    qdse_status s = set_params(c, p, rebuild);
    if (s != QDSE_OK) return s;
    if (!c->d_Kwhi) {
        cudaError_t e = dalloc(&c->d_Kwhi, (size_t)c->k_total);
        if (e == cudaSuccess) e = dalloc(&c->d_Kwlo, (size_t)c->k_total);
        if (e != cudaSuccess) return cuda_fail(c, e, "allocate omega-derivative kernels");
    }
    if (rebuild || !c->kw_valid) {
        QCHECK(c, launch_precompute(c, true), "precompute kernels and omega derivatives");
        QCHECK(c, launch_group_bands(c), "group bands");
        if (c->tc) QCHECK(c, launch_tc_extract(c), "tensor-core kernel planes");
        for (int b = 0; b < c->n_inst; ++b) c->k_omega[b] = p[b].omega;
        c->k_valid_for = 1;
        c->kw_valid = 1;
    }
    Ctl ctl = make_ctl(c);
    QCHECK(c, cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream), "ctl");
    // the adjoint applies at a fixed point: check F(x*) = x* first (relative residual 1e-6)
    QCHECK(c, launch_residual_fp64(c, A, B, c->work.xn64, c->work.xn64 + c->n_total, c->d_rel, 0,
                                   c->d_Khi, c->d_Klo),
           "fixed-point check");
    // mixed precision (FP32 inner sweeps, FP64 residuals) for MIXED/FP32 contexts on collocated
    // grids; plain FP64 successive approximation otherwise
    const bool mixed = (c->opt.precision == QDSE_MIXED || c->opt.precision == QDSE_FP32) &&
                       !c->any_staggered;
    QCHECK(c, launch_adjoint_init(c, c->work.lam, gA, gB, c->d_rel, 1e-6,
                                  mixed ? PH_RESID64 : PH_PICARD64),
           "adjoint init");
    QCHECK(c, launch_adjoint_prep(c, A, B), "adjoint prep");
    const auto t0 = std::chrono::steady_clock::now();
    bool timed_out = false;
    int chunk = 4;
    while (true) {
        for (int t = 0; t < chunk; ++t) {
            if (t == chunk - 1)
                QCHECK(c, cudaMemsetAsync(c->d_count, 0, sizeof(int), c->stream), "memset");
            if (mixed) {
                QCHECK(c, launch_adjoint_mixed_tick(c, gA, gB, c->d_count), "mixed adjoint tick");
                continue;
            }
            QCHECK(c, launch_adjoint_sweep(c, A, B, gA, gB), "transposed sweep");
            QCHECK(c, launch_adjoint_update(c, c->work.lam, c->work.lamn, c->d_count), "adjoint update");
        }
        QCHECK(c, cudaMemcpyAsync(c->h_count, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "poll");
        QCHECK(c, cudaStreamSynchronize(c->stream), "poll sync");
        c->polls++;
        if (*c->h_count == 0) break;
        if (c->opt.time_limit > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > c->opt.time_limit) {
            timed_out = true;
            break;
        }
        if (chunk < 64) chunk *= 2;
    }
    // dF/dD = (F(x*) - x0)/D and dF/domega at x*, both FP64 on the double-float kernels
    double* Fh = c->work.xn64;
    double* Fw = c->work.r64;
    QCHECK(c, launch_residual_fp64(c, A, B, Fh, Fh + c->n_total, nullptr, 1, c->d_Khi, c->d_Klo), "dF/dD");
    QCHECK(c, launch_residual_fp64(c, A, B, Fw, Fw + c->n_total, nullptr, 1, c->d_Kwhi, c->d_Kwlo), "dF/domega");
    QCHECK(c, launch_adjoint_grads(c, A, B, c->work.lam, Fh, Fw, g_params, inst_status), "gradients");
    if (lambda_out)
        QCHECK(c, cudaMemcpyAsync(lambda_out, c->work.lam, sizeof(double) * 2 * c->n_total,
                                  cudaMemcpyDeviceToDevice, c->stream), "copy lambda");
    QCHECK(c, cudaStreamSynchronize(c->stream), "sync");
    if (timed_out) return fail(c, QDSE_ERR_TIMEOUT, "time limit reached in the transposed solve");
    return QDSE_OK;
}

qdse_status qdse_condensate(qdse_ctx* c, const double* A, const double* B, double* out) {
    if (!c) return QDSE_ERR_ARG;
    if (!A || !B || !out) return fail(c, QDSE_ERR_ARG, "condensate: null pointer");
    QCHECK(c, launch_condensate(c, A, B, out), "condensate");
    return QDSE_OK;
}

qdse_status qdse_condensate_vjp(qdse_ctx* c, const double* A, const double* B,
                                const double* cbar, double* gA, double* gB) {
    if (!c) return QDSE_ERR_ARG;
    if (!A || !B || !cbar || !gA || !gB) return fail(c, QDSE_ERR_ARG, "condensate_vjp: null pointer");
    QCHECK(c, launch_condensate_vjp(c, A, B, cbar, gA, gB), "condensate vjp");
    return QDSE_OK;
}

qdse_status qdse_last_stats(const qdse_ctx* c, long long* kernel_launches, long long* fp32_sweeps,
                            long long* fp64_sweeps, long long* polls) {
    if (!c) return QDSE_ERR_ARG;
    unsigned long long ctr[4] = {0, 0, 0, 0};
    if (fp32_sweeps || fp64_sweeps) {
        cudaError_t e = cudaMemcpyAsync(ctr, c->d_sweeps, sizeof(ctr), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return QDSE_ERR_CUDA;
    }
    if (kernel_launches) *kernel_launches = c->launches;
    if (fp32_sweeps) *fp32_sweeps = (long long)ctr[0];
    if (fp64_sweeps) *fp64_sweeps = (long long)ctr[1];
    if (polls) *polls = c->polls;
    return QDSE_OK;
}

qdse_status qdse_last_work(const qdse_ctx* c, double* sweep_bytes, double* kernel_evals) {
    if (!c) return QDSE_ERR_ARG;
    unsigned long long ctr[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(ctr, c->d_sweeps, sizeof(ctr), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return QDSE_ERR_CUDA;
    if (sweep_bytes) *sweep_bytes = (double)ctr[2];
    if (kernel_evals) *kernel_evals = (double)ctr[3];
    return QDSE_OK;
}

qdse_status qdse_last_instance_stats(const qdse_ctx* c, long long* out, long long* out_cycles) {
    if (!c || !out) return QDSE_ERR_ARG;
    std::vector<DevState> st(c->n_inst);
    std::vector<unsigned long long> nnz(c->n_inst);
    cudaError_t e = cudaMemcpyAsync(st.data(), c->d_state, sizeof(DevState) * c->n_inst,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(nnz.data(), c->grid.nnz, sizeof(unsigned long long) * c->n_inst,
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return QDSE_ERR_CUDA;
    for (int b = 0; b < c->n_inst; ++b) {
        const DevState& s = st[b];
        out[5 * (size_t)b + 0] = s.iters - s.n64;
        out[5 * (size_t)b + 1] = s.n64;
        out[5 * (size_t)b + 2] = s.stall_max;
        out[5 * (size_t)b + 3] = c->k_valid_for ? (long long)nnz[b] : 0;
        out[5 * (size_t)b + 4] = s.phase;
        if (out_cycles) {
            out_cycles[2 * (size_t)b] = s.cyc_p;
            out_cycles[2 * (size_t)b + 1] = s.cyc_at;
        }
    }
    return QDSE_OK;
}

qdse_status qdse_set_profiling(qdse_ctx* c, int on) {
    if (!c) return QDSE_ERR_ARG;
    c->profiling = on ? 1 : 0;
    return QDSE_OK;
}

qdse_status qdse_profile(const qdse_ctx* c, double* ms, long long* launches) {
    if (!c || !ms || !launches) return QDSE_ERR_ARG;
    for (int k = 0; k < PK_COUNT; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return QDSE_ERR_CUDA;
    for (const auto& r : c->prof) {
        if (!r.a || !r.b || r.kind < 0 || r.kind >= PK_COUNT) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return QDSE_ERR_CUDA;
        ms[r.kind] += t;
        launches[r.kind] += 1;
    }
    return QDSE_OK;
}

}  // extern "C"
