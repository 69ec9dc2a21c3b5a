/*
 * qdse_mu.h -- C interface of libqdse for one sweep of the quark gap equation at finite quark
 * chemical potential mu, batched over many mu (Huang, Duan, Hu, Chen, arXiv:2012.03667, the
 * extension announced in Sec. V; the paper gives no equations for it).
 *
 * Equation solved (readings taken where the paper is silent):
 *   S^-1(p~) = i g_vec.p_vec A + i g_4 p~_4 C + B,  p~ = (p_vec, p_4 + i mu),  A, C, B complex
 *   functions of (|p_vec|, p_4);
 *   the gap equation of Sec. II (Eq. gendse) with p -> p~ in the propagator and the vertex, the
 *   gluon momentum k = p - q real, the interaction 8 pi^2 D/w^4 exp(-k^2/w^2) times the Landau
 *   projector (Eqs. KernelAnsatz, IRGsQC), colour factor cf;
 *   the Ball-Chiu vertex built from the Ward-Takahashi identity for this S^-1,
 *     Gamma_nu = Sigma_nu g_nu + t_nu (g_vec.t_vec dA/2 + g_4 t_4 dC/2 - i dB),  t = q~ + p~,
 *     Sigma_nu = (A_q + A_p)/2 for nu = 1..3, (C_q + C_p)/2 for nu = 4,
 *     dF = (F_q - F_p)/(q~^2 - p~^2)   (at mu = 0 with C = A: Eq. bcvtxmu with Eq. 2),
 *   or the bare vertex g_nu (QDSE_VERTEX_RL);
 *   projections A = tr[g_vec.p_vec S^-1]/(4 i p_vec^2), C = tr[g_4 S^-1]/(4 i p~_4),
 *   B = tr[S^-1]/4;  measure d^4q/(2 pi)^4 = 2 pi/(2 pi)^4 dq_4 |q_vec|^2 d|q_vec| dz.
 * One sweep maps the values at the external points and at the internal (quadrature) points to new
 * values at the external points.
 *
 * Finite temperature T (also named in Sec. V, without equations) uses the same calls: the internal
 * q_4 are the fermion Matsubara frequencies +-(2n + 1) pi T, the external p_4 axis is the positive
 * ones, and each frequency's weight in w_q carries 2 pi T in place of dq_4 (int dq_4/(2 pi) ->
 * T sum_n); mu then enters as p_4 -> (2n + 1) pi T + i mu.
 *
 * Conventions: as in qdse.h (GeV units; "device" pointers are device memory of the current CUDA
 * device, "host" pointers ordinary host memory; the caller owns every array passed in; work is
 * enqueued on the given stream, NULL = legacy default stream; the return value reports argument
 * and CUDA errors, qdse_mu_last_error() describes the last one; a grid is not thread-safe).
 * Complex arrays are interleaved (re, im) doubles, the layout of C99 double complex and of a
 * torch.complex128 tensor.
 */
#ifndef QDSE_MU_H
#define QDSE_MU_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qdse_mu_grid qdse_mu_grid; /* opaque: angular-moment table and workspaces */

/* Builds the grid and its angular-moment table on the device (enqueued on stream).
 * External points: n_ext pairs (p_abs[e] > 0, p4[e]), host double[n_ext] each.
 * Internal points: the product of n_r radial nodes q_abs (host double[n_r], > 0, strictly
 * increasing) and n_4 fourth components q4 (host double[n_4], strictly increasing); internal point
 * j = r * n_4 + f has |q_vec| = q_abs[r], q_4 = q4[f] and weight w_q[j] (host double[n_r * n_4]),
 * which must include |q_vec|^2 d|q_vec| dq_4.  Angular rule: n_z nodes z (host double[n_z], in
 * (-1, 1)) with weights w_z.  omega > 0: the interaction width (the table depends on it, on the
 * points and on the rule, not on D, m, mu or the colour factor).
 * precision: QDSE_FP64 (0) or QDSE_FP32 (3) -- the arithmetic of the sweeps; the moments are
 * always formed in FP64.
 * Pairs whose Gaussian exp(-((|p|-|q|)^2 + (p_4-q_4)^2)/omega^2) is below exp(-70) at every angle
 * are left out (a relative effect below 1e-30).
 * Returns QDSE_OK, QDSE_ERR_ARG (sizes < 1, non-finite or unordered nodes, omega <= 0,
 * precision), QDSE_ERR_OOM or QDSE_ERR_CUDA; *out is NULL unless QDSE_OK. */
int qdse_mu_grid_create(int n_ext, const double* p_abs, const double* p4, int n_r,
                        const double* q_abs, int n_4, const double* q4, const double* w_q, int n_z,
                        const double* z, const double* w_z, double omega, int precision,
                        void* stream, qdse_mu_grid** out);

/* As qdse_mu_grid_create, with the external points the product grid p_axis x p4_axis (host
 * double[n_pr], double[n_p4]; both > 0 and strictly increasing; external point e = i * n_p4 + k
 * has |p_vec| = p_axis[i], p_4 = p4_axis[k]).  Such a grid also carries the interpolation that
 * qdse_mu_solve uses to get A, C, B at the internal points (reading M6, the staggered-grid rule of
 * Sec. III along each axis): linear in |p| and in p_4 between the bracketing external nodes, held
 * at the first/last node outside them, and F(|q|, -q_4) = conj F(|q|, q_4) for q_4 < 0. */
int qdse_mu_grid_create_product(int n_pr, const double* p_axis, int n_p4, const double* p4_axis,
                                int n_r, const double* q_abs, int n_4, const double* q4,
                                const double* w_q, int n_z, const double* z, const double* w_z,
                                double omega, int precision, void* stream, qdse_mu_grid** out);

/* Successive approximation (Eq. jifen14 scheme) of the finite-mu equation for n_mu chemical
 * potentials at once: G = sweep(F, interpolate(F)); F <- G (alpha = 1) or (1 - alpha) F + alpha G.
 * Convergence (reading M7, per mu): max over A, C, B of max|F_new - F_old| / max|F_new| over the
 * grid (absolute where max|F_new| = 0) below tol; a converged mu is frozen while the others go on.
 * g: a product grid.  refine: NULL, or a product grid on the same points (normally QDSE_FP64 with
 * g QDSE_FP32): sweeps run on g until every mu's change is below max(tol, switch_tol), then on
 * refine until tol.  mu: host double[n_mu] (>= 0).  alpha in (0, 1].  max_iter >= 1 counts
 * sweeps of both phases.
 * F: device complex[n_mu][3][n_ext] -- the start on entry, the last iterate on return.
 * iters, status: host int[n_mu] or NULL -- sweeps to convergence (max_iter otherwise) and
 * QDSE_OK / QDSE_ERR_NOT_CONVERGED / QDSE_ERR_NONFINITE per mu.
 * Synchronises the stream once per sweep (to read the per-mu change).  Returns QDSE_OK unless an
 * argument or CUDA error occurred. */
int qdse_mu_solve(qdse_mu_grid* g, qdse_mu_grid* refine, int n_mu, const double* mu, double D,
                  double m, double cf, int vertex, double alpha, double tol, double switch_tol,
                  int max_iter, double* F, int* iters, int* status, void* stream);

/* Continuation in mu: qdse_mu_solve of all n_mu from F's starts, then up to max_rounds - 1 further
 * rounds in which every chemical potential that has not converged restarts from its nearest
 * converged neighbour in mu (the lower mu on a tie) -- all restarts of a round run as one batched
 * solve with max_iter sweeps.  A mu is not retried from the neighbour its previous attempt started
 * from; the rounds end when no mu has a new neighbour.  Near the chiral transition the Picard map
 * contracts slowly from a distant start; a converged neighbour puts the start on the same branch.
 * Arguments as qdse_mu_solve, plus max_rounds >= 1 (1: qdse_mu_solve alone).
 * F: a converged restart replaces the iterate; an unconverged one keeps the earlier attempt's.
 * iters: sweeps summed over the rounds; rounds: host int[n_mu] or NULL -- the round of the last
 * attempt (0 = the first solve).  Allocates one device buffer of n_mu solutions for the rounds.
 * Returns QDSE_OK unless an argument or CUDA error occurred. */
int qdse_mu_solve_continued(qdse_mu_grid* g, qdse_mu_grid* refine, int n_mu, const double* mu,
                            double D, double m, double cf, int vertex, double alpha, double tol,
                            double switch_tol, int max_iter, int max_rounds, double* F,
                            int* iters, int* status, int* rounds, void* stream);

/* Sizes: the pairs kept in the table and its device bytes (either pointer may be NULL). */
int qdse_mu_grid_info(const qdse_mu_grid* g, long long* n_pairs, long long* table_bytes);

/* One sweep for n_mu chemical potentials at once.
 * mu: host double[n_mu] (>= 0).  D, m, cf: interaction strength, current-quark mass, colour factor.
 * vertex: QDSE_VERTEX_BC or QDSE_VERTEX_RL.
 * F_ext: device complex[n_mu][3][n_ext] -- A, C, B at the external points for each mu (used in
 *        the vertex); F_int: device complex[n_mu][3][n_r * n_4] -- A, C, B at the internal points;
 * F_out: device complex[n_mu][3][n_ext] -- the new A, C, B; must not overlap the inputs.
 * An internal point with q~^2 = p~^2 (it coincides with an external point, or mu = 0 and equal
 * 4-radii) or a singular propagator gives non-finite output; no error is returned for it.
 * n_mu = 0 returns QDSE_OK without work.  The first call with a larger n_mu grows the grid's
 * workspace (a device allocation). */
int qdse_mu_sweep(qdse_mu_grid* g, int n_mu, const double* mu, double D, double m, double cf,
                  int vertex, const double* F_ext, const double* F_int, double* F_out,
                  void* stream);

/* Reading M8 (not in the paper; off by default): the Ball-Chiu vertex's difference numerators
 * F_q - F_p take, per (external p, internal q) pair, F_p + beta (F_ray - F_p) in place of F_p, where
 * F_ray is F interpolated (the rule of qdse_mu_grid_create_product) at the point where q~'s ray
 * crosses p~'s real 4-radius, (|q|, q_4) sqrt(|p|^2 + p_4^2)/sqrt(|q|^2 + q_4^2), and
 * beta = exp(-(2 mu |q_4 - p_4|/eta)^2).  As mu -> 0 the numerator then vanishes on the 4-sphere
 * q^2 = p^2 for any grid function, so the discrete principal-value sum of 1/(q~^2 - p~^2) no longer
 * couples F_p to itself; where 2 mu |q_4 - p_4| >> eta it is the exact quotient.  Applies to every
 * later qdse_mu_sweep and qdse_mu_solve on g (BC vertex).  g: a product grid; eta in GeV^2, > 0 turns
 * it on, 0 off.  Returns QDSE_OK or QDSE_ERR_ARG. */
int qdse_mu_set_ray_quotient(qdse_mu_grid* g, double eta);

/* Kernel timing.  With profiling on, every qdse_mu_sweep records CUDA events around its two
 * launches (the propagator prep and the sweep) on its stream, without synchronising.
 * qdse_mu_profile waits for the last recorded event, adds the elapsed times since the previous
 * read into ms[2] (prep, sweep; host double[2]) and the launch counts into launches[2] (host
 * long long[2]), and clears them.  Either output may be NULL.  Events accumulate (three per
 * sweep, reused after each read) until qdse_mu_profile is called; qdse_mu_solve's sweeps are
 * recorded too. */
int qdse_mu_set_profiling(qdse_mu_grid* g, int on);
int qdse_mu_profile(qdse_mu_grid* g, double* ms, long long* launches);

void qdse_mu_grid_destroy(qdse_mu_grid* g);

/* One-line description of the last error of a qdse_mu_* call on this thread. */
const char* qdse_mu_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QDSE_MU_H */
