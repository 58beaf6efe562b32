/*
 * pget.h -- C ABI of libpget.so, the GB300 (sm_103a) hot path of the Levenberg-Marquardt
 * reconstruction for passive gamma emission tomography (PGET).
 *
 * Paper: "Robust Model-Based Iteration for Passive Gamma Emission Tomography",
 * Heikkila, Heikkinen, Rimppi, Helin (arXiv 2604.26745).
 *
 * Unknowns: emission lambda and attenuation mu on an n x n pixel grid (pixel size 1,
 * row-major img[iy * n + ix], pixel centre at (ix - (n-1)/2, iy - (n-1)/2)).
 * Data: y[a * n_det + d], a = 0..n_angles-1 (phi_a = 2 pi a / n_angles), d = detector.
 *
 * Conventions shared by every call
 *   - Arrays are caller-owned, contiguous DEVICE pointers unless a name ends in _host.
 *     Element type: double for PGET_F64 and PGET_MIXED, float for PGET_F32 and
 *     PGET_F32_KAHAN.
 *     The library never frees caller memory and never keeps a caller pointer after a
 *     call returns, with one exception: a request queued by pget_submit reads the
 *     geometry-prior mask p->geo_mask while it runs.
 *   - stream is a cudaStream_t passed as void* (NULL: the legacy default stream).
 *     forward / jvp / vjp / reg_apply only enqueue work and return; they may reuse
 *     context workspace, so calls on one context must not overlap on different streams.
 *   - Every call returns a pget_status and never aborts, traps or prints.  On an error
 *     pget_last_error(ctx) gives a one-line message (thread-local, valid until the next
 *     call on that thread).
 *   - A context serves one device; it owns all workspace (allocated on first use for a
 *     geometry, freed by pget_destroy) and counts it against mem_budget_bytes.
 */
#ifndef PGET_H
#define PGET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PGET_OK = 0,
    PGET_EINVAL = 1,      /* bad argument: geometry, size, null pointer, precision      */
    PGET_ENOMEM = 2,      /* workspace would exceed the context's memory budget, or a   *
                           * host allocation failed                                      */
    PGET_EAGAIN = 3,      /* serving: no free slot or memory right now, retry later     */
    PGET_ECUDA = 4,       /* a CUDA runtime call failed (message has the CUDA error)    */
    PGET_ETIMEOUT = 5,    /* a bounded device-side wait ran out                         */
    PGET_ENUMERIC = 6,    /* NaN or Inf met in a result that must be finite             */
    PGET_ENOTFOUND = 7,   /* serving: unknown ticket                                     */
    PGET_EINTERNAL = 8    /* any other host-side failure inside the library (message)    */
} pget_status;

typedef enum {
    PGET_F64 = 0,         /* everything in double                                        */
    PGET_F32 = 1,         /* float ray sums and vectors; double dot products and scalars */
    PGET_F32_KAHAN = 2,   /* as PGET_F32 with Kahan-compensated sums along every ray     */
    PGET_MIXED = 3        /* the precision pattern of the solver: the Jacobian products of
                             CG (JVP and adjoint walks) as PGET_F32_KAHAN; the forward model
                             of every objective evaluation (the start of a solve and each
                             trial point, whose value decides acceptance) in double, and
                             the iterate, data, residuals, CG and LM vectors in double.
                             Caller arrays are double; the operator calls (pget_forward,
                             pget_jvp, pget_vjp) run the float walks.  Not taken by
                             pget_forward_noalloc or the batched operators. */
} pget_precision;

/* Measurement geometry (Sec. 2 and Sec. 2.1 of the paper: two opposed detector banks
 * with a half-pitch offset, a full rotation, collimated detectors).
 *   Detector d of bank b (b = 0: looks along theta = (cos phi, sin phi); b = 1: along
 *   theta + pi) sits at offset s_d = (d - (nb-1)/2 + b/2) * det_pitch in its bank's own
 *   frame, nb = n_det / n_banks.  Its collimator response is n_sub parallel sub-rays at
 *   offsets u_k with weights w_k (sum w = 1): triangular u_k = (k - (S-1)/2) 2p/(S+1),
 *   w_k ~ 1 - |u_k|/p; box u_k = (k - (S-1)/2) p/S, w_k = 1/S.
 *   A ray at offset s is sampled at x_j = s theta_perp + t_j theta, t_j = -r + (j+1/2) h,
 *   j = 0..T-1, T = ceil(2 r / h), theta_perp = (-sin, cos); the detector is at +theta. */
typedef struct {
    int32_t n;            /* grid size n >= 2                                             */
    int32_t n_angles;     /* 1..2^20, phi_a = 2 pi a / n_angles                          */
    int32_t n_det;        /* detectors in total, all banks                                */
    int32_t n_banks;      /* 1 or 2; 0 selects 2 when n_det == 182, else 1                */
    int32_t n_sub;        /* sub-rays per detector, 1..64                                 */
    int32_t collimator;   /* 0 box, 1 triangular                                          */
    double step;          /* ray sample spacing h in pixels (<= 0: 1)                     */
    double fov_radius;    /* r (<= 0: n / sqrt 2, the circumscribed disk of the grid)     */
    double det_pitch;     /* p (<= 0: 2 r / nb)                                           */
    /* Depth factors of Eq. (5) (optional; NULL: all ones): HOST arrays of T entries, T the
     * samples per ray (pget_geometry_info), copied when a call first uses the geometry.
     * Sample j of every sub-ray contributes h w_j lambda_j exp(-c_j E_j): depth_w[j] = w_j
     * >= 0 is the distance-dependent part of the detector response r_{m,n}, depth_c[j] =
     * c_j >= 0 the vertical-opening correction c_{m,n} of its attenuation (>= 1 in the
     * paper).  Not supported by pget_forward_noalloc. */
    const double* depth_w;
    const double* depth_c;
} pget_geometry;

/* Levenberg-Marquardt parameters (Sec. 2.2, Eq. (6)-(9), Sec. 3.1).
 * Objective f(u) = 1/2 |A(u) - y|^2 + R(lambda) + R(mu) with the smoothed total variation
 * R(v) = alpha sum_px sqrt(|grad v|^2 + tv_eps^2) (forward differences, zero-flux border);
 * tv_eps <= 0 selects the quadratic R(v) = alpha/2 |grad v|^2. */
typedef struct {
    double alpha_lambda, alpha_mu;   /* prior weights (1e-2)                                     */
    double tv_eps;                   /* smoothing of the TV prior (1e-3); <= 0: quadratic prior  */
    double lambda_max, mu_max;       /* box [0, lambda_max] x [0, mu_max] (2.0, 0.2)             */
    int32_t max_iters;               /* LM iterations; a rejected trial counts as one (20)       */
    int32_t cg_max_iters;            /* CG iterations per LM step (30)                           */
    double cg_rel_tol;               /* CG stops when |res| <= tol |rhs| (1e-6)                  */
    double nu0_scale;                /* nu_0 = nu0_scale |J g|^2 / |g|^2, g = grad f(u_0) (1e-3) */
    double nu_up, nu_down;           /* nu *= nu_up if rho < rho_lo, *= nu_down if rho > rho_hi  */
    double eta;                      /* accept iff rho > eta, eta in (0, 1/4) (1e-3)             */
    double rho_lo, rho_hi;           /* (0.25, 0.75)                                              */
    double nu_min, nu_max;           /* nu clamped to [nu_min nu_0, nu_max nu_0] (1e-12, 1e12)   */
    int32_t precision;               /* pget_precision                                           */
    int32_t alpha_decay_iters;       /* continuation (Sec. 3.1): iteration k uses the prior       */
    double alpha_decay;              /* weights alpha / alpha_decay^min(k, alpha_decay_iters);   */
                                     /* f and its gradient are re-evaluated when they change.    */
                                     /* alpha_decay <= 1 or 0 iterations: fixed alpha (1.0, 0)   */
    /* geometry priors of Eq. (6), added to R: geo_alpha_lambda |(1 - M) lambda|^2 +
     * geo_alpha_mu |(1 - M)(mu - geo_mu_water)|^2 with M = geo_mask, the [n][n] mask of the
     * potential rod locations in [0, 1] (device memory, element type of the precision;
     * caller-owned, must stay valid for the call).  NULL: no geometry prior (default).
     * The continuation above scales these weights too. */
    double geo_alpha_lambda, geo_alpha_mu, geo_mu_water;
    const void* geo_mask;
    /* inner solver of the LM step (Sec. 2.2): 0 = CG on Eq. (9), then projection of
     * u + delta onto the constraint set (default); 1 = gradient projection on the
     * constrained subproblem (the scaled gradient projection the paper names, identity
     * scaling, Barzilai-Borwein lengths, exact line search), capped by cg_max_iters and
     * stopped when the unit-step projected gradient falls below cg_rel_tol times its
     * first value */
    int32_t inner_solver;
    /* linear bound of the constraint set (Sec. 2.2: no strongly emitting pixel of low
     * attenuation): 1 adds lambda <= lin_slope mu + lin_offset per pixel to the box
     * (lin_slope, lin_offset >= 0, finite); 0 = box only (default).  Every projection
     * (start, step, gradient projection, proposals) is then the Euclidean projection of
     * each pixel's pair (lambda, mu) onto the polygon box & bound. */
    int32_t lin_constraint;
    double lin_slope, lin_offset;
} pget_lm_params;

#define PGET_TRACE 256

typedef struct {
    int32_t iters_run, accepted, cg_iters_total;
    int32_t status;                  /* pget_status of the solve                             */
    double f0, f_final, nu0, nu_final;
    /* per iteration k < min(iters_run, PGET_TRACE): objective after the iteration, rho,
     * nu after its update, model decrease m(0) - m(s), actual decrease, accepted flag,
     * CG iterations run */
    double f[PGET_TRACE], rho[PGET_TRACE], nu[PGET_TRACE], pred[PGET_TRACE], ared[PGET_TRACE];
    int32_t acc[PGET_TRACE], cg_iters[PGET_TRACE];
    double device_ms;                /* device time of the solve (CUDA events)               */
} pget_lm_report;

typedef struct pget_ctx pget_ctx;

/* Create a context on `device` whose workspace may use at most mem_budget_bytes
 * (0: no limit).  *ctx is set to NULL on failure. */
pget_status pget_create(pget_ctx** ctx, int device, size_t mem_budget_bytes);

/* Free the context and all of its workspace (waits for its work to finish). */
pget_status pget_destroy(pget_ctx* ctx);

/* Fill *out with the defaults listed above (precision PGET_F32_KAHAN). */
void pget_default_params(pget_lm_params* out);

/* Forward model y = A(lambda, mu): the attenuated ray transform of Eq. (1) in its
 * sampled form (Eq. (5)): per ray q = h sum_j lambda_j exp(-E_j),
 * E_j = h (mu_j / 2 + sum_{i > j} mu_i) (i > j: nearer the detector), lambda_j, mu_j
 * bilinear samples (zero outside the grid), y = sum_k w_k q_k.
 * lam, mu: [n][n] in; y: [n_angles][n_det] out. */
pget_status pget_forward(pget_ctx* ctx, const pget_geometry* g, int32_t precision,
                         const void* lam, const void* mu, void* y, void* stream);

/* Jacobian-vector product dy = J (dlam, dmu), the Frechet derivative of Eq. (2):
 * per ray q' = h sum_j exp(-E_j) (dlam_j - lambda_j dE_j), dE_j = h (dmu_j/2 + sum_{i>j} dmu_i).
 * lam, mu, dlam, dmu: [n][n] in; dy: [n_angles][n_det] out. */
pget_status pget_jvp(pget_ctx* ctx, const pget_geometry* g, int32_t precision,
                     const void* lam, const void* mu, const void* dlam, const void* dmu,
                     void* dy, void* stream);

/* Adjoint product (glam, gmu) = J^T r (the F'* of Thm. 3.1 and the convergence proof in
 * Sec. 3.1), computed as a gather: every output pixel sums the contributions of the ray
 * samples whose bilinear footprint covers it; no atomics, deterministic.
 * lam, mu: [n][n] in; r: [n_angles][n_det] in; glam, gmu: [n][n] out. */
pget_status pget_vjp(pget_ctx* ctx, const pget_geometry* g, int32_t precision,
                     const void* lam, const void* mu, const void* r, void* glam, void* gmu,
                     void* stream);

/* The three operators above for a batch of independent image pairs of one geometry
 * (the differentiation workload: many (lambda, mu) pairs per call): item b of lam, mu
 * ([batch][n][n]), dlam, dmu ([batch][n][n]), y, dy, r ([batch][n_angles][n_det]) and glam,
 * gmu ([batch][n][n]) is the single-item call's argument, and its result equals the
 * single-item call's bitwise.  The items run in chunks, each chunk one walk launch over all
 * its items' views (the chunk holds up to 4 GiB of adjoint partial images, so at least one
 * item); the chunk buffers stay with the context for the next call.  Precisions PGET_F64,
 * PGET_F32 and PGET_F32_KAHAN (PGET_EINVAL otherwise); batch = 0 does nothing.
 * Asynchronous like the single-item calls. */
pget_status pget_forward_batch(pget_ctx* ctx, const pget_geometry* g, int32_t precision, int32_t batch,
                               const void* lam, const void* mu, void* y, void* stream);
pget_status pget_jvp_batch(pget_ctx* ctx, const pget_geometry* g, int32_t precision, int32_t batch,
                           const void* lam, const void* mu, const void* dlam, const void* dmu, void* dy,
                           void* stream);
pget_status pget_vjp_batch(pget_ctx* ctx, const pget_geometry* g, int32_t precision, int32_t batch,
                           const void* lam, const void* mu, const void* r, void* glam, void* gmu,
                           void* stream);

/* Device-side status of the asynchronous operator calls above (pget_forward, pget_jvp,
 * pget_vjp) made on this context since the last call of this function or since the
 * geometry or precision last changed.  Waits for `stream`, reads the kernels' error word
 * and clears it: PGET_OK; PGET_ETIMEOUT when a chunk copy of a walk did not arrive within
 * its wait limit (the outputs of that call are void); PGET_ECUDA when an adjoint stencil
 * bound was violated (never expected: the geometry guarantees it).  This is how a caller
 * checks results those calls could not check without waiting for the device.  The
 * paper has no counterpart. */
pget_status pget_operator_status(pget_ctx* ctx, void* stream);

/* Prior of the objective above (it stands in for the P1/P2 terms of Eq. (6)):
 * out = alpha grad^T W(u) grad v with the lagged-diffusivity weights
 * W(u) = 1 / sqrt(|grad u|^2 + eps^2) (eps <= 0: W = 1), and, when value_host is not
 * NULL, *value_host = R(u) (synchronises the stream).  With v = u, out is grad R(u).
 * u, v, out: [n][n]. */
pget_status pget_reg_apply(pget_ctx* ctx, int32_t n, int32_t precision, double alpha,
                           double eps, const void* u, const void* v, void* out,
                           double* value_host, void* stream);

/* Conjugate gradients from x = 0 on the damped normal equations of Eq. (9):
 * (J^T J + alpha grad^T W grad + nu I) x = rhs at u = (lam, mu), W frozen at u,
 * stopping after p->cg_max_iters iterations or when |res| <= p->cg_rel_tol |rhs|.
 * rhs, x: [2][n][n] (lambda block, then mu block).  *iters_host (optional) gets the
 * iterations run (synchronises the stream). */
pget_status pget_cg_solve(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                          const void* lam, const void* mu, double nu, const void* rhs,
                          void* x, int32_t* iters_host, void* stream);

/* Initial guess (the paper states none): mu = mu_init, lambda = c with
 * c = sum y / sum A(1, mu_init), both projected onto the box. */
pget_status pget_initial_guess(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                               double mu_init, const void* y, void* lam, void* mu, void* stream);

/* Levenberg-Marquardt trust-region solve (Sec. 2.2 and 3.1): each iteration runs CG on
 * Eq. (9) (or gradient projection, inner_solver), takes s = P(u + delta) - u with P the
 * projection onto the constraint set (the box, and the linear bound if set), evaluates the
 * model decrease of Eq. (8) and rho of Eq. (12), accepts iff rho > eta and updates nu.
 * All state stays on the device: the whole solve (every iteration, with device-side
 * flags for the CG exit and the acceptance) is one CUDA graph, captured on the first call
 * with these parameters and replayed afterwards; one host synchronisation at the end reads
 * the FP64 scalars and traces into the report.  lam_io, mu_io: initial guess in, result
 * out.  rep: host memory.  Blocks until done. */
pget_status pget_lm_solve(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                          const void* y, void* lam_io, void* mu_io, pget_lm_report* rep,
                          void* stream);

/* ---- safeguarded acceleration (Prop. conv_check and Alg. 2, Sec. 3.1) ----
 *
 * Alg. 2 lets a learned operator G propose u~ = G(u_k, s_k) after every LM step s_k and
 * keeps u~ only if it passes the paper's convergence check.  The two calls below are
 * the library side of that loop; the proposal itself comes from the caller (any model). */

/* Scalars of one trust-region trial (host memory). */
typedef struct {
    double f;        /* f(u) = 1/2 |A(u) - y|^2 + R(u)                                 */
    double pred;     /* m_k(0) - m_k(s_k), Eq. (8)                                        */
    double ared;     /* f(u) - f(u + s_k)                                                  */
    double rho;      /* Eq. (12); -inf when pred <= 0 or f(u + s_k) is not finite          */
    double nu_next;  /* nu after the schedule (x nu_up if rho < rho_lo, x nu_down if
                        rho > rho_hi), not clamped: the caller clamps with its own nu_0   */
    double nu0;      /* the damping used when nu <= 0 was passed, else 0                  */
    int32_t accept;  /* rho > eta                                                          */
    int32_t cg_iters;
} pget_trial_report;

/* One trust-region trial of the LM iteration at the feasible point u = (lam, mu) with
 * damping nu (nu <= 0: nu_0 = nu0_scale |J g|^2 / |g|^2 at u, as a solve starts): CG on
 * Eq. (9), s_k = P(u + delta) - u (P: projection onto the constraint set), model and actual
 * decrease, rho, acceptance.  u is
 * not changed (this is the s_k = LMA(u_k) of Alg. 2).  s_out: [2][n][n] device, the step.
 * rep: host.  Synchronises the stream. */
pget_status pget_lm_trial(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                          const void* y, const void* lam, const void* mu, double nu,
                          void* s_out, pget_trial_report* rep, void* stream);

/* Result of the convergence check for one proposal (host memory). */
typedef struct {
    double f;          /* f(u)                                                */
    double pred_step;  /* m_k(0) - m_k(s_k) of the LM step                    */
    double pred_prop;  /* m_k(0) - m_k(s~) of the proposal's step             */
    double ared_prop;  /* f(u) - f(u + s~)                                    */
    double rho_prop;   /* rho(s~), -inf when pred_prop <= 0                   */
    int32_t accept;    /* rho(s~) > eta and m_k(s~) <= m_k(s_k)               */
    int32_t pad;
} pget_check_report;

/* The check of Prop. conv_check / Alg. 2 for the proposal u~ = (prop_lam, prop_mu) at the
 * feasible point u with the LM step s_step ([2][n][n], as pget_lm_trial returns it):
 * s~ = P(u~) - u (the proposal is projected onto the constraint set like the LM step),
 * then accept iff rho(s~) > p->eta and m_k(s~) <= m_k(s_k).  The caller then sets
 * u_{k+1} = P(u~) when accepted (pget_project), else u + s_k if the trial accepted, else
 * u.  All
 * arrays device [n][n] (s_step [2][n][n]); rep: host.  Synchronises the stream. */
pget_status pget_proposal_check(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                                const void* y, const void* lam, const void* mu,
                                const void* s_step, const void* prop_lam, const void* prop_mu,
                                pget_check_report* rep, void* stream);

/* Outcome of one iteration of Alg. 2 after its proposal check (host memory). */
typedef struct {
    pget_check_report check;  /* the check of the proposal; zero when none was given            */
    int32_t checked;          /* 1 when a proposal was given and checked                         */
    int32_t took;             /* the new iterate: 0 u_k (nothing accepted), 1 u_k + s_k (the LM
                                 step), 2 P(u~) (the proposal)                                    */
    double nu_next;           /* damping of iteration k + 1: the trial's nu_next clamped to
                                 [nu_min nu0, nu_max nu0], as a plain solve clamps it            */
} pget_step_report;

/* One iteration of the accelerated scheme (Alg. 2) after its LM trial: with the trial's
 * step s_step ([2][n][n] device) and report `trial` at the feasible point (lam_io, mu_io),
 * checks the proposal u~ = (prop_lam, prop_mu) (device [n][n]; both NULL: no proposal) by
 * Prop. conv_check (rho(s~) > eta and m_k(s~) <= m_k(s_k), as pget_proposal_check) and
 * replaces (lam_io, mu_io) in place by the next iterate: P(u~) if the proposal passes,
 * else P(u_k + s_k) if the trial was accepted, else u_k unchanged (P: projection onto the
 * constraint set; u_k + s_k is feasible already, the projection only rounds).  The
 * parameters of iteration k follow the continuation of Sec. 3.1 (pget_params_at(p, k));
 * nu0 is the first damping of the solve (the trial of iteration 0 reports it).  The
 * paper's Alg. 2 leaves the damping after an accepted proposal open: the trial's rho
 * drives it, as in a plain solve.  rep: host.  Synchronises the stream. */
pget_status pget_lm_step_with_proposal(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                                       int32_t k, const void* y, void* lam_io, void* mu_io,
                                       const void* s_step, const pget_trial_report* trial, double nu0,
                                       const void* prop_lam, const void* prop_mu, pget_step_report* rep,
                                       void* stream);

/* The parameters of LM iteration k under the continuation of Sec. 3.1 (host only): the
 * prior weights (TV and geometry priors) divided by alpha_decay^min(k, alpha_decay_iters),
 * everything else copied; fixed weights when alpha_decay <= 1 or alpha_decay_iters = 0.
 * pget_lm_solve uses the same schedule.  PGET_EINVAL for null pointers or k < 0. */
pget_status pget_params_at(const pget_lm_params* p, int32_t k, pget_lm_params* out);

/* Validate LM parameters on the host, without a context: PGET_OK, or PGET_EINVAL with a
 * message naming the field (NaN or out-of-range values, unknown precision or options).
 * Every call that takes parameters runs the same check first. */
pget_status pget_check_params(const pget_lm_params* p);

/* Derived sizes of a geometry (any output pointer may be NULL; host only, no context):
 * samples per ray T of the discretised ray integral of Eq. (5) (the length of the depth
 * tables), detector banks and pitch p of the device of Sec. 2, field-of-view radius r,
 * and distinct rays per view (slots).  PGET_EINVAL for an invalid geometry. */
pget_status pget_geometry_info(const pget_geometry* g, int32_t* n_samples, int32_t* n_banks, double* fov_radius,
                               double* det_pitch, int32_t* max_slots);

/* Launch plans of the three ray operators (forward A of Eq. (1), J of Eq. (2) and its
 * adjoint) for a geometry and precision, as every call on that pair will use them.  Index
 * 0 forward, 1 JVP, 2 adjoint: image rows staged per chunk, chunks per view, dynamic
 * shared memory per CTA.  adjoint_phases: the adjoint's accumulation scheme, 0 for per-ray
 * 4-column stencils gathered per pixel, K > 0 for K phase-coloured row buffers (slot t
 * writes buffer t mod K; rays of one phase never touch the same pixel, so each buffer is
 * written without conflicts and a pixel sums its K buffers).  Host only, no context;
 * PGET_EINVAL for a null argument, an unknown precision or an invalid geometry. */
typedef struct pget_walk_plan_info {
    int32_t threads;            /* threads per CTA (one per distinct ray of a view) */
    int32_t rows_per_chunk[3];
    int32_t chunks[3];
    int32_t smem_bytes[3];
    int32_t adjoint_phases;
    int32_t phases_needed;      /* phases the slot lattice needs (the plan takes phase
                                   buffers when at most 16 are needed and they fit; 0: a
                                   degenerate lattice) */
} pget_walk_plan_info;
pget_status pget_walk_plans(const pget_geometry* g, int32_t precision, pget_walk_plan_info* out);

/* Projection onto the constraint set of p (Sec. 2.2): every pixel's pair (lambda, mu)
 * is replaced, in place, by its Euclidean projection onto the box [0, lambda_max] x
 * [0, mu_max], intersected with lambda <= lin_slope mu + lin_offset when p->lin_constraint
 * is set.  lam, mu: [n][n] device arrays in the element type of p->precision (caller-
 * owned).  Asynchronous on the stream; PGET_EINVAL for null pointers, n < 1 or invalid
 * parameters. */
pget_status pget_project(pget_ctx* ctx, const pget_lm_params* p, int32_t n, void* lam, void* mu, void* stream);

/* The LM solve of Sec. 2.2 and 3.1, as pget_lm_solve, with HOST buffers (pinned or
 * pageable) in the element type of p->precision: copies y_host to the device,
 * computes the initial guess (mu_init 0.01) when init_guess != 0 (else takes
 * lam_host / mu_host as the initial guess), solves, and copies the result back. */
pget_status pget_lm_solve_host(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p,
                               const void* y_host, void* lam_host, void* mu_host,
                               int32_t init_guess, pget_lm_report* rep, void* stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of reconstructions (the LM solve of Sec. 2.2 and 3.1 per request;
 * the paper has no serving layer): each accepted request gets an in-flight slot
 * (its own workspace, stream and captured LM graph, all state on the device); requests
 * that arrive while others run are admitted as soon as a slot and device memory are
 * free, and their kernels overlap on the GPU with those of the requests in flight.
 * Results are identical to pget_lm_solve on the same inputs (the kernels are
 * deterministic and a slot shares nothing with other slots).
 *
 * pget_submit: y ([n_angles][n_det]) and the optional initial guess lam0, mu0 ([n][n];
 *   both NULL: the pget_initial_guess reading with mu_init 0.01) are device pointers in
 *   the element type of p->precision; they are copied into slot memory before the call
 *   returns, so the caller may free them afterwards; so are the geometry's depth tables.
 *   The parameters are taken by value, except p->geo_mask, which the request reads while it
 *   runs: keep that array valid until pget_poll reports done.  Returns PGET_EAGAIN when every slot
 *   is busy or the memory budget of the context is in use (retry after a poll),
 *   PGET_ENOMEM when the request can never fit the budget, PGET_EINVAL for bad
 *   arguments.  Up to 8 requests are in flight (environment PGET_MAX_INFLIGHT, <= 64).
 * pget_poll: *done = 0 while the request runs; when it has finished, copies the result
 *   into lam_out / mu_out (device, may be NULL), fills *rep (host, may be NULL), frees the
 *   slot and sets *done = 1.  PGET_ENOTFOUND for an unknown or already collected ticket.
 * pget_cancel: drops a request (its queued kernels finish first; they cannot be aborted).
 * pget_inflight: number of occupied slots. */
pget_status pget_submit(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* y,
                        const void* lam0, const void* mu0, uint64_t* ticket);
pget_status pget_poll(pget_ctx* ctx, uint64_t ticket, void* lam_out, void* mu_out, pget_lm_report* rep,
                      int* done);
pget_status pget_cancel(pget_ctx* ctx, uint64_t ticket);
int32_t pget_inflight(pget_ctx* ctx);

/* ------------------------------------------------------ allocation-free forward
 * The forward model of Eq. (1) in its discrete form Eq. (5), as pget_forward computes it.
 * The paper has no counterpart to this entry point; it serves callers that are not allowed to
 * allocate device memory (a host framework whose allocator owns the GPU, allocation-free
 * real-time sections, processes with a memory budget fixed up front), which cannot use
 * the context-based calls above because a pget_ctx obtains its workspace with cudaMalloc.
 *
 * pget_forward_noalloc computes exactly what pget_forward computes, on the current
 * device, without a context.  All of its scratch (geometry tables and the packed image
 * layouts) lives in one fixed array of 8 MiB in device memory, defined in the library and
 * held by every device that loads it until the process exits.
 *   - A geometry whose scratch exceeds 8 MiB returns PGET_ENOMEM before any work is
 *     queued (2 * (n+2)^2 image elements of 8 or 16 bytes plus 8 bytes per ray slot and
 *     view; e.g. n = 128 with 360 angles x 182 detectors x 5 sub-rays needs about 2 MiB).
 *   - Bad arguments return PGET_EINVAL, CUDA failures PGET_ECUDA, a host-side failure
 *     (a failed mutex) PGET_EINTERNAL.  Errors are reported by the status only:
 *     pget_last_error is not updated (storing a message could allocate).
 *   - The first call on a device looks up the array's device address and caches it; make
 *     that first call before any stream capture.  The call refuses to run while `stream`
 *     is being captured into a CUDA graph (PGET_EINVAL): its table copy reads a host
 *     staging buffer shared by all calls, which a replay would read later.
 *   - Every call overwrites the same array (image borders are cleared on each call), and
 *     the tables are built in one host staging buffer for the whole process.  Calls that
 *     overlapped on the GPU, or built their tables at the same time, would race; to
 *     prevent that, each call holds one process-wide lock from building its tables until
 *     its projection has finished, so concurrent calls (several host threads, one device
 *     or several) run one after another.
 *   - The call waits for its projection (it synchronises `stream`) and reads the kernel's
 *     error word: PGET_ETIMEOUT when a chunk copy did not arrive within its wait limit
 *     (y is then void), PGET_ECUDA for any other device-side condition.
 *   - The call allocates no device or host memory (the per-device tables of shared-memory
 *     permissions and kernel variants it consults are fixed arrays).
 * lam, mu: [n][n] device in; y: [n_angles][n_det] device out; stream as above. */
pget_status pget_forward_noalloc(const pget_geometry* g, int32_t precision, const void* lam,
                                 const void* mu, void* y, void* stream);

/* ------------------------------------------------------------- diagnostics
 * Device time of the hot kernels, measured with CUDA events recorded on the stream each
 * kernel is launched on (no effect on results).  pget_profile_enable resets the counters;
 * pget_profile_read synchronises on the recorded events and fills up to max entries
 * (walk_forward, walk_jvp, walk_vjp, reduce_views), returning how many were written. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} pget_kernel_stat;

pget_status pget_profile_enable(pget_ctx* ctx, int32_t enable);
int32_t pget_profile_read(pget_ctx* ctx, pget_kernel_stat* out, int32_t max);

/* Kernel launches issued by this library since it was loaded (all contexts). */
long long pget_launch_count(void);

/* Message of the last error on this thread ("" if none). */
const char* pget_last_error(pget_ctx* ctx);

/* Library version string. */
const char* pget_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PGET_H */
