/*
 * pget_oracle.c -- plain FP64 CPU oracle for the PGET Levenberg-Marquardt hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: "Robust Model-Based Iteration for Passive Gamma Emission Tomography",
 * Heikkila, Heikkinen, Rimppi, Helin (arXiv 2604.26745).
 *
 * What is computed, function by function (all arithmetic in double):
 *   og_forward   -- the attenuated ray transform of Sec. 2.1, Eq. (1), sampled along
 *                   straight rays as the discrete model of Eq. (5): every map value is
 *                   a bilinear sample of the pixel grid at the ray point (the paper
 *                   rotates the maps per projection; bilinear sampling on the rotated
 *                   lattice is that rotation), the beam transform B mu is the sum of
 *                   the samples nearer the detector plus half of the own sample, and
 *                   the detector reading is the collimator-weighted mean of sub-rays.
 *   og_jvp       -- the exact derivative of og_forward, i.e. the Frechet derivative
 *                   of Eq. (2): D_lambda F[dl] = F(dl, mu), D_mu F[dm] = -F(lambda B dm, mu).
 *   og_vjp       -- the adjoint of og_jvp (used as F'* in Thm. 3.1 and the proof of the
 *                   convergence proposition, Sec. 3.1), written as a scatter loop.
 *   og_reg_*     -- the regulariser that replaces the P1/P2 terms of Eq. (6):
 *                   alpha * sum sqrt(|grad u|^2 + eps^2) (smoothed TV), its gradient
 *                   alpha grad^T W grad u and the frozen-weight Hessian alpha grad^T W grad;
 *                   optionally with the geometry priors of Eq. (6) themselves,
 *                   alpha_1 |P1 lambda|^2 + alpha_2 |P2 mu|^2 (og_geo_*).
 *   og_cg        -- conjugate gradients on the damped normal equations of Eq. (9):
 *                   (J^T J + alpha grad^T W grad + nu I) delta = rhs.
 *   og_sgp       -- gradient projection on the box-constrained form of Eq. (9), the
 *                   inner solver Sec. 2.2 names (scaled gradient projection, identity
 *                   scaling, Barzilai-Borwein lengths, exact line search).
 *   og_project   -- projection onto the constraint set of Eq. (6): the box, and with
 *                   lin_constraint the per-pixel linear bound lambda <= k mu + b.
 *   og_lm        -- the trust-region LM iteration of Sec. 2.2: step from Eq. (9),
 *                   projection onto the constraint set, model m_k of Eq. (8), agreement
 *                   ratio rho of Eq. (12), acceptance rho > eta with eta in (0, 1/4);
 *                   optionally with the continuation alpha^(k) = alpha / 5^k of Sec. 3.1.
 *   og_lm_trial  -- one trial of that iteration at a given point and damping, returning
 *                   the step s_k without moving the iterate (the LMA(u_k) of Alg. 2).
 *   og_check_proposal -- the safeguard of Prop. conv_check / Alg. 2 (Sec. 3.1): accept a
 *                   proposal u~ iff rho(s~) > eta and m_k(s~) <= m_k(s_k).
 *
 * Pins: every function above is checked by tests/test_oracle_*.py against closed
 * forms, hand-computed values, finite differences, the adjoint identity, dense
 * linear algebra and the monotone decrease the paper proves (Sec. 3.1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ geometry */

typedef struct {
    int32_t n;           /* image is n x n pixels of unit size                       */
    int32_t n_angles;    /* phi_a = 2 pi a / n_angles                                 */
    int32_t n_det;       /* detectors in total (all banks)                            */
    int32_t n_banks;     /* 1, or 2 opposed banks (0: 2 if n_det == 182 else 1)       */
    int32_t n_sub;       /* sub-rays per detector (collimator response samples)       */
    int32_t collimator;  /* 0 box, 1 triangular                                       */
    double step;         /* ray sample spacing h (0: 1)                               */
    double fov_radius;   /* r_Omega (0: n / sqrt 2)                                   */
    double det_pitch;    /* p (0: 2 r_Omega / detectors per bank)                     */
    int32_t interleave;  /* 1: bank B shifted by p/2 (default); 0: no shift (test aid) */
    /* depth factors of Eq. (5) over the sample index j of every ray (length T, or NULL
     * for all ones): depth_w[j] scales the emission of sample j (the part of the
     * detector response r_{m,n} that varies with the distance to the detector), depth_c[j]
     * its attenuation exponent (the vertical-opening correction c_{m,n} >= 1) */
    const double* depth_w;
    const double* depth_c;
} og_geom;

typedef struct {
    og_geom g;
    int nb;       /* detectors per bank */
    int T;        /* samples per ray    */
    double h, r, p, c;  /* step, fov radius, pitch, pixel-centre offset (n-1)/2 */
} og_ctx;

/* Fill defaults and validate. Returns 0 on success, 1 on a bad geometry. */
static int og_setup(const og_geom* in, og_ctx* o) {
    memset(o, 0, sizeof *o);
    o->g = *in;
    og_geom* g = &o->g;
    if (g->n < 2 || g->n_angles < 1 || g->n_det < 1 || g->n_sub < 1) return 1;
    if (g->collimator != 0 && g->collimator != 1) return 1;
    if (g->n_banks == 0) g->n_banks = (g->n_det == 182) ? 2 : 1;
    if (g->n_banks != 1 && g->n_banks != 2) return 1;
    if (g->n_det % g->n_banks) return 1;
    o->nb = g->n_det / g->n_banks;
    o->h = g->step > 0 ? g->step : 1.0;
    o->r = g->fov_radius > 0 ? g->fov_radius : g->n / sqrt(2.0);
    o->p = g->det_pitch > 0 ? g->det_pitch : 2.0 * o->r / o->nb;
    o->T = (int)ceil(2.0 * o->r / o->h);
    o->c = 0.5 * (g->n - 1);
    return 0;
}

/* Collimator response as parallel sub-rays: offset u_k and weight w_k, sum w = 1. */
static void og_subrays(const og_ctx* o, double* u, double* w) {
    int S = o->g.n_sub;
    double tot = 0.0;
    for (int k = 0; k < S; ++k) {
        double m = k - 0.5 * (S - 1);
        if (o->g.collimator == 1) {
            u[k] = m * 2.0 * o->p / (S + 1);
            w[k] = 1.0 - fabs(u[k]) / o->p;
        } else {
            u[k] = m * o->p / S;
            w[k] = 1.0;
        }
        tot += w[k];
    }
    for (int k = 0; k < S; ++k) w[k] /= tot;
}

/* One ray: direction theta = (cos psi, sin psi), normal (-sin psi, cos psi), offset s.
 * Bank b looks along phi + b*pi; its detectors sit at (d - (nb-1)/2 + b/2) p. */
typedef struct { double ct, st, s; } og_ray;

static og_ray og_make_ray(const og_ctx* o, int a, int bank, int d, double u) {
    og_ray ry;
    double psi = 2.0 * M_PI * a / o->g.n_angles + bank * M_PI;
    ry.ct = cos(psi);
    ry.st = sin(psi);
    double shift = (bank == 1 && o->g.interleave) ? 0.5 : 0.0;
    ry.s = (d - 0.5 * (o->nb - 1) + shift) * o->p + u;
    return ry;
}

/* Ray point j: x = s theta_perp + t_j theta, t_j = -r + (j + 1/2) h.  Returns the
 * pixel-index coordinates (fx, fy) of that point. */
static void og_point(const og_ctx* o, const og_ray* ry, int j, double* fx, double* fy) {
    double t = -o->r + (j + 0.5) * o->h;
    double x1 = -ry->s * ry->st + t * ry->ct;
    double x2 = ry->s * ry->ct + t * ry->st;
    *fx = x1 + o->c;
    *fy = x2 + o->c;
}

/* The four bilinear neighbours of (fx, fy) with their weights; neighbours outside the
 * grid get index -1 (their value is zero).  Returns 0 if all four are outside. */
static int og_bilinear(const og_ctx* o, double fx, double fy, int idx[4], double wt[4]) {
    int n = o->g.n;
    double fl_x = floor(fx), fl_y = floor(fy);
    if (fl_x < -1.0 || fl_x > n - 1 || fl_y < -1.0 || fl_y > n - 1) return 0;
    int ix = (int)fl_x, iy = (int)fl_y;
    double ax = fx - fl_x, ay = fy - fl_y;
    int xs[4] = {ix, ix + 1, ix, ix + 1};
    int ys[4] = {iy, iy, iy + 1, iy + 1};
    double ws[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};
    int any = 0;
    for (int q = 0; q < 4; ++q) {
        if (xs[q] >= 0 && xs[q] < n && ys[q] >= 0 && ys[q] < n) {
            idx[q] = ys[q] * n + xs[q];
            any = 1;
        } else {
            idx[q] = -1;
        }
        wt[q] = ws[q];
    }
    return any;
}

static double og_sample(const double* img, const int idx[4], const double wt[4]) {
    double v = 0.0;
    for (int q = 0; q < 4; ++q)
        if (idx[q] >= 0) v += wt[q] * img[idx[q]];
    return v;
}

/* ------------------------------------------------------------- forward model */

/* depth factors of sample j (1 without tables) */
static double og_dw(const og_ctx* o, int j) { return o->g.depth_w ? o->g.depth_w[j] : 1.0; }
static double og_dc(const og_ctx* o, int j) { return o->g.depth_c ? o->g.depth_c[j] : 1.0; }

/* Ray sum of Eq. (1) on one ray: q = h sum_j w_j lambda_j exp(-c_j E_j),
 * E_j = h (mu_j / 2 + sum_{i > j} mu_i), i > j being nearer the detector, with the depth
 * factors w_j, c_j of Eq. (5) (1 by default). */
static double og_ray_sum(const og_ctx* o, const og_ray* ry, const double* lam, const double* mu) {
    double h = o->h, S = 0.0, q = 0.0;
    for (int j = o->T - 1; j >= 0; --j) {
        double fx, fy;
        int idx[4];
        double wt[4];
        og_point(o, ry, j, &fx, &fy);
        if (!og_bilinear(o, fx, fy, idx, wt)) continue;
        double l = og_sample(lam, idx, wt), m = og_sample(mu, idx, wt);
        double E = h * (S + 0.5 * m);
        q += h * og_dw(o, j) * l * exp(-og_dc(o, j) * E);
        S += m;
    }
    return q;
}

int og_forward(const og_geom* gin, const double* lam, const double* mu, double* y) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    int S = o.g.n_sub;
    double* u = malloc(sizeof(double) * S);
    double* w = malloc(sizeof(double) * S);
    og_subrays(&o, u, w);
    int total = o.g.n_angles * o.g.n_det;
#pragma omp parallel for schedule(dynamic, 4)
    for (int ad = 0; ad < total; ++ad) {
        int a = ad / o.g.n_det, dd = ad % o.g.n_det;
        int bank = dd / o.nb, d = dd % o.nb;
        double acc = 0.0;
        for (int k = 0; k < S; ++k) {
            og_ray ry = og_make_ray(&o, a, bank, d, u[k]);
            acc += w[k] * og_ray_sum(&o, &ry, lam, mu);
        }
        y[ad] = acc;
    }
    free(u);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------ JVP */

/* Derivative of og_ray_sum along (dl, dm), Eq. (2):
 * q' = h sum_j w_j exp(-c_j E_j) (dl_j - lambda_j c_j dE_j), dE_j = h (dm_j / 2 + sum_{i > j} dm_i). */
static double og_ray_jvp(const og_ctx* o, const og_ray* ry, const double* lam, const double* mu,
                         const double* dl, const double* dm) {
    double h = o->h, S = 0.0, dS = 0.0, q = 0.0;
    for (int j = o->T - 1; j >= 0; --j) {
        double fx, fy;
        int idx[4];
        double wt[4];
        og_point(o, ry, j, &fx, &fy);
        if (!og_bilinear(o, fx, fy, idx, wt)) continue;
        double l = og_sample(lam, idx, wt), m = og_sample(mu, idx, wt);
        double a = og_sample(dl, idx, wt), b = og_sample(dm, idx, wt);
        double E = h * (S + 0.5 * m);
        double dE = h * (dS + 0.5 * b);
        double c = og_dc(o, j);
        q += h * og_dw(o, j) * exp(-c * E) * (a - l * c * dE);
        S += m;
        dS += b;
    }
    return q;
}

int og_jvp(const og_geom* gin, const double* lam, const double* mu, const double* dl,
           const double* dm, double* dy) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    int S = o.g.n_sub;
    double* u = malloc(sizeof(double) * S);
    double* w = malloc(sizeof(double) * S);
    og_subrays(&o, u, w);
    int total = o.g.n_angles * o.g.n_det;
#pragma omp parallel for schedule(dynamic, 4)
    for (int ad = 0; ad < total; ++ad) {
        int a = ad / o.g.n_det, dd = ad % o.g.n_det;
        int bank = dd / o.nb, d = dd % o.nb;
        double acc = 0.0;
        for (int k = 0; k < S; ++k) {
            og_ray ry = og_make_ray(&o, a, bank, d, u[k]);
            acc += w[k] * og_ray_jvp(&o, &ry, lam, mu, dl, dm);
        }
        dy[ad] = acc;
    }
    free(u);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------ VJP */

/* Adjoint of og_ray_jvp for one ray with residual weight rho, scattered into gl, gm:
 *   d q / d lambda_j = h w_j exp(-c_j E_j)
 *   d q / d mu_i     = -h Q_i,  Q_i = sum_{j < i} c_j t_j + c_i t_i / 2,  t_j = h w_j lambda_j exp(-c_j E_j)
 * (j < i: farther from the detector), each spread to pixels by the bilinear weights. */
static void og_ray_vjp(const og_ctx* o, const og_ray* ry, const double* lam, const double* mu,
                       double rho, double* gl, double* gm, double* ex, double* lv) {
    double h = o->h, S = 0.0;
    int T = o->T;
    /* pass 1, detector side first: attenuation factors and emission samples */
    for (int j = T - 1; j >= 0; --j) {
        double fx, fy;
        int idx[4];
        double wt[4];
        og_point(o, ry, j, &fx, &fy);
        if (!og_bilinear(o, fx, fy, idx, wt)) {
            ex[j] = 0.0;
            lv[j] = 0.0;
            continue;
        }
        double l = og_sample(lam, idx, wt), m = og_sample(mu, idx, wt);
        ex[j] = og_dw(o, j) * exp(-og_dc(o, j) * h * (S + 0.5 * m));  /* w_j exp(-c_j E_j) */
        lv[j] = l;
        S += m;
    }
    /* pass 2, far side first: Q prefix and the scatter */
    double P = 0.0;
    for (int j = 0; j < T; ++j) {
        double fx, fy;
        int idx[4];
        double wt[4];
        og_point(o, ry, j, &fx, &fy);
        if (!og_bilinear(o, fx, fy, idx, wt)) continue;
        double c = og_dc(o, j);
        double term = h * lv[j] * ex[j];
        double Q = P + 0.5 * c * term;
        double vl = rho * h * ex[j];
        double vm = -rho * h * Q;
        for (int q = 0; q < 4; ++q) {
            if (idx[q] < 0) continue;
            gl[idx[q]] += wt[q] * vl;
            gm[idx[q]] += wt[q] * vm;
        }
        P += c * term;
    }
}

/* Angle chunks of the VJP scatter.  The chunks are summed in order, so the result does
 * not depend on the thread count; changing the chunk count only changes the summation
 * order (a rounding-level change used by the tests to measure rounding sensitivity). */
static int og_vjp_chunks = 32;

void og_set_vjp_chunks(int c) { og_vjp_chunks = c > 0 ? c : 32; }

int og_vjp(const og_geom* gin, const double* lam, const double* mu, const double* r,
           double* gl, double* gm) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    int S = o.g.n_sub, np = o.g.n * o.g.n, T = o.T;
    double* u = malloc(sizeof(double) * S);
    double* w = malloc(sizeof(double) * S);
    og_subrays(&o, u, w);
    int nch = o.g.n_angles < og_vjp_chunks ? o.g.n_angles : og_vjp_chunks;
    /* one private image pair per fixed angle chunk, summed in chunk order: the result
     * does not depend on the thread count */
    double* part = calloc((size_t)nch * 2 * np, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int ch = 0; ch < nch; ++ch) {
        double* pl = part + (size_t)ch * 2 * np;
        double* pm = pl + np;
        double* ex = malloc(sizeof(double) * T);
        double* lv = malloc(sizeof(double) * T);
        int a0 = (int)((long)o.g.n_angles * ch / nch), a1 = (int)((long)o.g.n_angles * (ch + 1) / nch);
        for (int a = a0; a < a1; ++a)
            for (int dd = 0; dd < o.g.n_det; ++dd) {
                int bank = dd / o.nb, d = dd % o.nb;
                double rv = r[a * o.g.n_det + dd];
                for (int k = 0; k < S; ++k) {
                    og_ray ry = og_make_ray(&o, a, bank, d, u[k]);
                    og_ray_vjp(&o, &ry, lam, mu, w[k] * rv, pl, pm, ex, lv);
                }
            }
        free(ex);
        free(lv);
    }
    for (int i = 0; i < np; ++i) {
        double sl = 0.0, sm = 0.0;
        for (int ch = 0; ch < nch; ++ch) {
            sl += part[(size_t)ch * 2 * np + i];
            sm += part[(size_t)ch * 2 * np + np + i];
        }
        gl[i] = sl;
        gm[i] = sm;
    }
    free(part);
    free(u);
    free(w);
    return 0;
}

/* ------------------------------------------------------------ regulariser */

/* Forward differences with a zero-flux boundary: gx = u[x+1] - u[x] (0 on the last
 * column), gy = u[y+1] - u[y] (0 on the last row). */
static void og_grad(int n, const double* u, double* gx, double* gy) {
    for (int iy = 0; iy < n; ++iy)
        for (int ix = 0; ix < n; ++ix) {
            int i = iy * n + ix;
            gx[i] = (ix < n - 1) ? u[i + 1] - u[i] : 0.0;
            gy[i] = (iy < n - 1) ? u[i + n] - u[i] : 0.0;
        }
}

/* Adjoint of og_grad: out = grad^T (gx, gy). */
static void og_grad_t(int n, const double* gx, const double* gy, double* out) {
    for (int iy = 0; iy < n; ++iy)
        for (int ix = 0; ix < n; ++ix) {
            int i = iy * n + ix;
            double v = 0.0;
            if (ix < n - 1) v -= gx[i];
            if (ix > 0) v += gx[i - 1];
            if (iy < n - 1) v -= gy[i];
            if (iy > 0) v += gy[i - n];
            out[i] = v;
        }
}

/* Lagged-diffusivity weights W = 1 / sqrt(|grad u|^2 + eps^2); eps <= 0 gives W = 1
 * (the quadratic smoothness prior). */
void og_reg_weights(int n, double eps, const double* u, double* W) {
    int np = n * n;
    double* gx = malloc(sizeof(double) * np);
    double* gy = malloc(sizeof(double) * np);
    og_grad(n, u, gx, gy);
    for (int i = 0; i < np; ++i)
        W[i] = (eps > 0) ? 1.0 / sqrt(gx[i] * gx[i] + gy[i] * gy[i] + eps * eps) : 1.0;
    free(gx);
    free(gy);
}

/* Value R(u) = alpha sum sqrt(|grad u|^2 + eps^2)  (eps > 0)
 *           or alpha/2 sum |grad u|^2              (eps <= 0). */
double og_reg_value(int n, double alpha, double eps, const double* u) {
    int np = n * n;
    double* gx = malloc(sizeof(double) * np);
    double* gy = malloc(sizeof(double) * np);
    og_grad(n, u, gx, gy);
    double v = 0.0;
    for (int i = 0; i < np; ++i) {
        double s2 = gx[i] * gx[i] + gy[i] * gy[i];
        v += (eps > 0) ? sqrt(s2 + eps * eps) : 0.5 * s2;
    }
    free(gx);
    free(gy);
    return alpha * v;
}

/* out = alpha grad^T diag(W) grad v.  With W from og_reg_weights(u) and v = u this is
 * the gradient of og_reg_value at u; for other v it is the frozen-weight Hessian. */
void og_reg_apply(int n, double alpha, const double* W, const double* v, double* out) {
    int np = n * n;
    double* gx = malloc(sizeof(double) * np);
    double* gy = malloc(sizeof(double) * np);
    og_grad(n, v, gx, gy);
    for (int i = 0; i < np; ++i) {
        gx[i] *= W[i];
        gy[i] *= W[i];
    }
    og_grad_t(n, gx, gy, out);
    for (int i = 0; i < np; ++i) out[i] *= alpha;
    free(gx);
    free(gy);
}

/* ------------------------------------------------------------------- CG */

typedef struct {
    double alpha_lambda, alpha_mu, tv_eps;
    double lambda_max, mu_max;
    int32_t max_iters, cg_max_iters;
    double cg_rel_tol;
    double nu0_scale, nu_up, nu_down, eta, rho_lo, rho_hi, nu_min, nu_max;
    int32_t alpha_decay_iters, pad;
    double alpha_decay;
    double geo_alpha_lambda, geo_alpha_mu, geo_mu_water;
    const double* geo_mask;  /* [n][n] potential rod locations in [0, 1], or NULL */
    int32_t inner_solver;    /* 0: CG on Eq. (9) then projection; 1: gradient projection */
    int32_t lin_constraint;  /* 1: add the per-pixel linear bound lambda <= lin_slope mu + lin_offset */
    double lin_slope, lin_offset;
} og_params;

/* Geometry priors of Eq. (6): alpha_1 |P1 lambda|^2 + alpha_2 |P2 mu|^2 with the
 * projections P1 lambda = (1 - M) lambda and P2 mu = (1 - M)(mu - mu_water), M the mask of
 * the potential rod locations (values outside them are penalised; water keeps its
 * attenuation).  Quadratic: gradient 2 alpha (1 - M)^2 (u - c), Hessian 2 alpha (1 - M)^2. */
static double og_geo_value(int n, const og_params* pr, const double* lam, const double* mu) {
    if (!pr->geo_mask) return 0.0;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < n * n; ++i) {
        double om = 1.0 - pr->geo_mask[i];
        double pl = om * lam[i], pm = om * (mu[i] - pr->geo_mu_water);
        a += pl * pl;
        b += pm * pm;
    }
    return pr->geo_alpha_lambda * a + pr->geo_alpha_mu * b;
}

/* grad += gradient of the geometry priors at (lam, mu) (stacked [lambda; mu]) */
static void og_geo_grad_add(int n, const og_params* pr, const double* lam, const double* mu, double* grad) {
    if (!pr->geo_mask) return;
    int np = n * n;
    for (int i = 0; i < np; ++i) {
        double om2 = (1.0 - pr->geo_mask[i]) * (1.0 - pr->geo_mask[i]);
        grad[i] += 2.0 * pr->geo_alpha_lambda * om2 * lam[i];
        grad[np + i] += 2.0 * pr->geo_alpha_mu * om2 * (mu[i] - pr->geo_mu_water);
    }
}

/* out += Hessian of the geometry priors times the stacked vector v */
static void og_geo_hess_add(int n, const og_params* pr, const double* v, double* out) {
    if (!pr->geo_mask) return;
    int np = n * n;
    for (int i = 0; i < np; ++i) {
        double om2 = (1.0 - pr->geo_mask[i]) * (1.0 - pr->geo_mask[i]);
        out[i] += 2.0 * pr->geo_alpha_lambda * om2 * v[i];
        out[np + i] += 2.0 * pr->geo_alpha_mu * om2 * v[np + i];
    }
}

/* s^T (Hessian of the geometry priors) s */
static double og_geo_quad(int n, const og_params* pr, const double* s) {
    if (!pr->geo_mask) return 0.0;
    int np = n * n;
    double q = 0.0;
    for (int i = 0; i < np; ++i) {
        double om2 = (1.0 - pr->geo_mask[i]) * (1.0 - pr->geo_mask[i]);
        q += 2.0 * om2 * (pr->geo_alpha_lambda * s[i] * s[i] + pr->geo_alpha_mu * s[np + i] * s[np + i]);
    }
    return q;
}

/* Prior weights of LM iteration k under the continuation of Sec. 3.1 (alpha^(k) =
 * alpha / decay^k, the decrease halted after alpha_decay_iters iterations); decay <= 1
 * or no iterations: fixed alpha. */
static og_params og_params_at(const og_params* pr, int k) {
    og_params q = *pr;
    if (pr->alpha_decay > 1.0 && pr->alpha_decay_iters > 0) {
        int e = k < pr->alpha_decay_iters ? k : pr->alpha_decay_iters;
        double sc = pow(pr->alpha_decay, -(double)e);
        q.alpha_lambda *= sc;
        q.alpha_mu *= sc;
        q.geo_alpha_lambda *= sc;
        q.geo_alpha_mu *= sc;
    }
    return q;
}

static double og_dot(int m, const double* a, const double* b) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

/* out = (J^T J + H + nu I) v for the stacked vector v = (v_lambda, v_mu). */
static void og_normal_apply(const og_geom* g, const og_params* pr, const double* lam,
                            const double* mu, const double* Wl, const double* Wm, double nu,
                            const double* v, double* out, double* tmp_y, double* tmp_img) {
    int n = g->n, np = n * n;
    og_jvp(g, lam, mu, v, v + np, tmp_y);
    og_vjp(g, lam, mu, tmp_y, out, out + np);
    og_reg_apply(n, pr->alpha_lambda, Wl, v, tmp_img);
    for (int i = 0; i < np; ++i) out[i] += tmp_img[i] + nu * v[i];
    og_reg_apply(n, pr->alpha_mu, Wm, v + np, tmp_img);
    for (int i = 0; i < np; ++i) out[np + i] += tmp_img[i] + nu * v[np + i];
    og_geo_hess_add(n, pr, v, out);
}

/* Plain CG from x = 0 on (J^T J + H + nu I) x = b, the normal equations of Eq. (9).
 * Stops after cg_max iterations or when |res| <= tol |b|.  Returns iterations run. */
int og_cg(const og_geom* g, const og_params* pr, const double* lam, const double* mu,
          const double* Wl, const double* Wm, double nu, const double* b, double* x) {
    og_ctx o;
    if (og_setup(g, &o)) return -1;
    int np = o.g.n * o.g.n, m = 2 * np;
    double* res = malloc(sizeof(double) * m);
    double* p = malloc(sizeof(double) * m);
    double* q = malloc(sizeof(double) * m);
    double* ty = malloc(sizeof(double) * o.g.n_angles * o.g.n_det);
    double* ti = malloc(sizeof(double) * np);
    memset(x, 0, sizeof(double) * m);
    memcpy(res, b, sizeof(double) * m);
    memcpy(p, b, sizeof(double) * m);
    double rr = og_dot(m, res, res);
    double bnorm = sqrt(rr);
    int it = 0;
    if (bnorm > 0.0) {
        for (it = 0; it < pr->cg_max_iters;) {
            og_normal_apply(&o.g, pr, lam, mu, Wl, Wm, nu, p, q, ty, ti);
            double pq = og_dot(m, p, q);
            if (!(pq > 0.0)) break;
            double a = rr / pq;
            for (int i = 0; i < m; ++i) {
                x[i] += a * p[i];
                res[i] -= a * q[i];
            }
            ++it;
            double rr_new = og_dot(m, res, res);
            if (sqrt(rr_new) <= pr->cg_rel_tol * bnorm) break;
            double beta = rr_new / rr;
            rr = rr_new;
            for (int i = 0; i < m; ++i) p[i] = res[i] + beta * p[i];
        }
    }
    free(res);
    free(p);
    free(q);
    free(ty);
    free(ti);
    return it;
}

static double og_clamp(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Euclidean projection of one pixel's pair (lambda, mu) onto the constraint set of
 * Sec. 2.2: the box [0, lambda_max] x [0, mu_max] and, with lin_constraint, the linear
 * bound lambda <= k mu + b (k = lin_slope >= 0, b = lin_offset >= 0: no strongly emitting
 * pixel with low attenuation).  The set is a convex polygon.  If the box projection meets
 * the linear bound it is the answer (the nearest point of a larger set, lying in the
 * smaller one).  Otherwise the bound is active at the answer, which is then the nearest
 * point of the segment of the line lambda = k t + b, mu = t that lies in the box:
 * t = ((lambda - b) k + mu) / (k^2 + 1) (the foot of the perpendicular), clamped to
 * 0 <= t <= mu_max and k t + b <= lambda_max. */
static void og_project_px(const og_params* pr, double* l, double* m) {
    double pl = og_clamp(*l, 0.0, pr->lambda_max), pm = og_clamp(*m, 0.0, pr->mu_max);
    if (pr->lin_constraint && pl - pr->lin_slope * pm > pr->lin_offset) {
        double k = pr->lin_slope, b = pr->lin_offset;
        double t = ((*l - b) * k + *m) / (k * k + 1.0);
        double t_hi = pr->mu_max;
        if (k > 0.0 && (pr->lambda_max - b) / k < t_hi) t_hi = (pr->lambda_max - b) / k;
        t = og_clamp(t, 0.0, t_hi);
        pl = k * t + b;
        pm = t;
    }
    *l = pl;
    *m = pm;
}

/* Projection of a pair of images (in place). */
void og_project(const og_params* pr, int np, double* lam, double* mu) {
    for (int i = 0; i < np; ++i) og_project_px(pr, &lam[i], &mu[i]);
}

/* Gradient projection for the box-constrained LM subproblem of Sec. 2.2 (the scaled
 * gradient projection method the paper cites, with the identity scaling):
 *   min_s q(s) = <g, s> + 1/2 s^T (J^T J + H + nu I) s   subject to  u + s in the box,
 * from s = 0.  Iteration: d = P(u + s - alpha grad q(s)) - u - s; exact line search on
 * [0, 1] for the quadratic q along d; alpha alternates the two Barzilai-Borwein lengths
 * |d|^2 / <d, A d> and <d, A d> / |A d|^2, clamped to [1e-10, 1e10].  Stops after
 * cg_max_iters iterations or when the unit-step projected gradient
 * |P(u + s - grad q) - u - s| <= cg_rel_tol times its value at s = 0.  P is the projection
 * onto the box.
 * With lin_constraint P projects onto the box and the linear bound (og_project_px).
 * Returns iterations run; s_out is feasible (u + s in the constraint set). */
int og_sgp(const og_geom* g, const og_params* pr, const double* lam, const double* mu,
           const double* Wl, const double* Wm, double nu, const double* grad_f, double* s_out) {
    og_ctx o;
    if (og_setup(g, &o)) return -1;
    int np = o.g.n * o.g.n, m = 2 * np;
    double* x = s_out;
    double* gq = malloc(sizeof(double) * m);
    double* d = malloc(sizeof(double) * m);
    double* Ad = malloc(sizeof(double) * m);
    double* ty = malloc(sizeof(double) * o.g.n_angles * o.g.n_det);
    double* ti = malloc(sizeof(double) * np);
    memset(x, 0, sizeof(double) * m);
    memcpy(gq, grad_f, sizeof(double) * m);
    double alpha = 1.0, pg0 = -1.0;
    int it = 0;
    for (it = 0; it < pr->cg_max_iters;) {
        /* unit-step projected gradient (stopping measure) and the projected step */
        double pg = 0.0;
        for (int i = 0; i < np; ++i) {
            double z1l = lam[i] + x[i] - gq[i], z1m = mu[i] + x[np + i] - gq[np + i];
            og_project_px(pr, &z1l, &z1m);
            z1l -= lam[i] + x[i];
            z1m -= mu[i] + x[np + i];
            pg += z1l * z1l + z1m * z1m;
            double zl = lam[i] + x[i] - alpha * gq[i], zm = mu[i] + x[np + i] - alpha * gq[np + i];
            og_project_px(pr, &zl, &zm);
            d[i] = zl - lam[i] - x[i];
            d[np + i] = zm - mu[i] - x[np + i];
        }
        pg = sqrt(pg);
        if (pg0 < 0.0) pg0 = pg;
        if (pg <= pr->cg_rel_tol * pg0 || pg0 == 0.0) break;
        double gd = og_dot(m, gq, d);
        if (!(gd < 0.0)) break;
        og_normal_apply(&o.g, pr, lam, mu, Wl, Wm, nu, d, Ad, ty, ti);
        double dAd = og_dot(m, d, Ad);
        if (!(dAd > 0.0)) break;
        double lstep = -gd / dAd;
        if (lstep > 1.0) lstep = 1.0;
        for (int i = 0; i < m; ++i) {
            x[i] += lstep * d[i];
            gq[i] += lstep * Ad[i];
        }
        ++it;
        double a_next = (it % 2) ? og_dot(m, d, d) / dAd : dAd / og_dot(m, Ad, Ad);
        alpha = og_clamp(a_next, 1e-10, 1e10);
    }
    free(gq);
    free(d);
    free(Ad);
    free(ty);
    free(ti);
    return it;
}

/* ------------------------------------------------------------------- LM */

#define OG_TRACE 256

typedef struct {
    int32_t iters_run, accepted, cg_iters_total, status;
    double f0, f_final, nu0, nu_final;
    double f[OG_TRACE], rho[OG_TRACE], nu[OG_TRACE], pred[OG_TRACE], ared[OG_TRACE];
    int32_t acc[OG_TRACE], cg_iters[OG_TRACE];
} og_report;

/* f(u) = 1/2 |A(u) - y|^2 + R_lambda + R_mu (Eq. (6) with the smoothed-TV prior);
 * writes the residual r = A(u) - y. */
static double og_objective(const og_geom* g, const og_params* pr, const double* lam,
                           const double* mu, const double* y, double* r) {
    int m = g->n_angles * g->n_det;
    og_forward(g, lam, mu, r);
    for (int i = 0; i < m; ++i) r[i] -= y[i];
    return 0.5 * og_dot(m, r, r) + og_reg_value(g->n, pr->alpha_lambda, pr->tv_eps, lam) +
           og_reg_value(g->n, pr->alpha_mu, pr->tv_eps, mu) + og_geo_value(g->n, pr, lam, mu);
}

/* Gradient of the objective at u: grad = J^T r + alpha grad^T W grad u. */
static void og_gradient(const og_geom* g, const og_params* pr, const double* lam,
                        const double* mu, const double* r, const double* Wl, const double* Wm,
                        double* grad, double* tmp) {
    int np = g->n * g->n;
    og_vjp(g, lam, mu, r, grad, grad + np);
    og_reg_apply(g->n, pr->alpha_lambda, Wl, lam, tmp);
    for (int i = 0; i < np; ++i) grad[i] += tmp[i];
    og_reg_apply(g->n, pr->alpha_mu, Wm, mu, tmp);
    for (int i = 0; i < np; ++i) grad[np + i] += tmp[i];
    og_geo_grad_add(g->n, pr, lam, mu, grad);
}


/* Levenberg-Marquardt trust-region iteration, Sec. 2.2 and Sec. 3.1:
 *   delta from CG on (J^T J + H + nu I) delta = -grad            (Eq. (9), nu = beta_k)
 *   s = P_C(u + delta) - u      (constraint set of Eq. (6): the box, and the linear bound if set)
 *   m_k(0) - m_k(s) = -<s, grad> - |J s|^2 / 2 - s^T H s / 2      (Eq. (8))
 *   rho = (f(u) - f(u + s)) / (m_k(0) - m_k(s))                   (Eq. (12))
 *   accept iff rho > eta; nu <- nu_up nu if rho < rho_lo, nu <- nu nu_down if rho > rho_hi.
 * lam, mu hold the initial guess on entry (projected onto the constraint set) and the result
 * on exit. */
int og_lm(const og_geom* gin, const og_params* pr, const double* y, double* lam, double* mu,
          og_report* rep) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    const og_geom* g = &o.g;
    int n = g->n, np = n * n, m = g->n_angles * g->n_det;
    memset(rep, 0, sizeof *rep);
    double* r = malloc(sizeof(double) * m);
    double* rt = malloc(sizeof(double) * m);
    double* Js = malloc(sizeof(double) * m);
    double* Wl = malloc(sizeof(double) * np);
    double* Wm = malloc(sizeof(double) * np);
    double* grad = malloc(sizeof(double) * 2 * np);
    double* rhs = malloc(sizeof(double) * 2 * np);
    double* delta = malloc(sizeof(double) * 2 * np);
    double* s = malloc(sizeof(double) * 2 * np);
    double* ut = malloc(sizeof(double) * 2 * np);
    double* tmp = malloc(sizeof(double) * np);
    double* Hs = malloc(sizeof(double) * np);

    og_project(pr, np, lam, mu);
    double f = og_objective(g, pr, lam, mu, y, r);
    og_reg_weights(n, pr->tv_eps, lam, Wl);
    og_reg_weights(n, pr->tv_eps, mu, Wm);
    og_gradient(g, pr, lam, mu, r, Wl, Wm, grad, tmp);
    rep->f0 = f;

    /* nu_0 = nu0_scale |J g|^2 / |g|^2 */
    double gg = og_dot(2 * np, grad, grad);
    double nu0 = 1.0;
    if (gg > 0.0) {
        og_jvp(g, lam, mu, grad, grad + np, Js);
        nu0 = pr->nu0_scale * og_dot(m, Js, Js) / gg;
    }
    if (!(nu0 > 0.0)) nu0 = 1.0;
    double nu = nu0;
    rep->nu0 = nu0;

    int k;
    const og_params* pr0 = pr;
    og_params prk = og_params_at(pr0, 0);
    for (k = 0; k < pr0->max_iters; ++k) {
        /* continuation: a new alpha changes f and its gradient at the current iterate */
        og_params next = og_params_at(pr0, k);
        if (k > 0 && (next.alpha_lambda != prk.alpha_lambda || next.alpha_mu != prk.alpha_mu)) {
            prk = next;
            f = og_objective(g, &prk, lam, mu, y, r);
            og_gradient(g, &prk, lam, mu, r, Wl, Wm, grad, tmp);
        }
        pr = &prk;
        int it;
        if (pr->inner_solver == 1) {  /* gradient projection: delta is already feasible */
            it = og_sgp(g, pr, lam, mu, Wl, Wm, nu, grad, delta);
        } else {
            for (int i = 0; i < 2 * np; ++i) rhs[i] = -grad[i];
            it = og_cg(g, pr, lam, mu, Wl, Wm, nu, rhs, delta);
        }
        rep->cg_iters_total += it;
        /* projected step */
        for (int i = 0; i < np; ++i) {
            ut[i] = lam[i] + delta[i];
            ut[np + i] = mu[i] + delta[np + i];
            og_project_px(pr, &ut[i], &ut[np + i]);
            s[i] = ut[i] - lam[i];
            s[np + i] = ut[np + i] - mu[i];
        }
        /* predicted decrease of the Gauss-Newton model */
        og_jvp(g, lam, mu, s, s + np, Js);
        double sHs = 0.0;
        og_reg_apply(n, pr->alpha_lambda, Wl, s, Hs);
        sHs += og_dot(np, s, Hs);
        og_reg_apply(n, pr->alpha_mu, Wm, s + np, Hs);
        sHs += og_dot(np, s + np, Hs);
        sHs += og_geo_quad(n, pr, s);
        double pred = -og_dot(2 * np, s, grad) - 0.5 * og_dot(m, Js, Js) - 0.5 * sHs;
        /* actual decrease */
        double ft = og_objective(g, pr, ut, ut + np, y, rt);
        double ared = f - ft;
        double rho = (pred > 0.0 && isfinite(ft)) ? ared / pred : -INFINITY;
        int accept = rho > pr->eta;
        if (accept) {
            memcpy(lam, ut, sizeof(double) * np);
            memcpy(mu, ut + np, sizeof(double) * np);
            memcpy(r, rt, sizeof(double) * m);
            f = ft;
            og_reg_weights(n, pr->tv_eps, lam, Wl);
            og_reg_weights(n, pr->tv_eps, mu, Wm);
            og_gradient(g, pr, lam, mu, r, Wl, Wm, grad, tmp);
            rep->accepted++;
        }
        if (rho < pr->rho_lo)
            nu *= pr->nu_up;
        else if (rho > pr->rho_hi)
            nu *= pr->nu_down;
        nu = og_clamp(nu, pr->nu_min * nu0, pr->nu_max * nu0);
        if (k < OG_TRACE) {
            rep->f[k] = f;
            rep->rho[k] = rho;
            rep->nu[k] = nu;
            rep->pred[k] = pred;
            rep->ared[k] = ared;
            rep->acc[k] = accept;
            rep->cg_iters[k] = it;
        }
    }
    pr = pr0;
    rep->iters_run = k;
    rep->f_final = f;
    rep->nu_final = nu;
    free(r);
    free(rt);
    free(Js);
    free(Wl);
    free(Wm);
    free(grad);
    free(rhs);
    free(delta);
    free(s);
    free(ut);
    free(tmp);
    free(Hs);
    return 0;
}

/* ------------------------------------------------- safeguarded acceleration */

typedef struct {
    double f, pred, ared, rho, nu_next, nu0;
    int32_t accept, cg_iters;
} og_trial;

typedef struct {
    double f, pred_step, pred_prop, ared_prop, rho_prop;
    int32_t accept, pad;
} og_check;

/* m_k(0) - m_k(s) at u for the stacked step s (Eq. (8) with the prior's frozen-weight
 * Hessian): -<s, grad> - |J s|^2 / 2 - s^T H s / 2. */
static double og_model_decrease(const og_geom* g, const og_params* pr, const double* lam,
                                const double* mu, const double* grad, const double* Wl,
                                const double* Wm, const double* s, double* Js, double* Hs) {
    int n = g->n, np = n * n, m = g->n_angles * g->n_det;
    og_jvp(g, lam, mu, s, s + np, Js);
    double sHs = 0.0;
    og_reg_apply(n, pr->alpha_lambda, Wl, s, Hs);
    sHs += og_dot(np, s, Hs);
    og_reg_apply(n, pr->alpha_mu, Wm, s + np, Hs);
    sHs += og_dot(np, s + np, Hs);
    sHs += og_geo_quad(n, pr, s);
    return -og_dot(2 * np, s, grad) - 0.5 * og_dot(m, Js, Js) - 0.5 * sHs;
}

/* One trust-region trial of the LM iteration at the feasible point u = (lam, mu) with
 * damping nu (nu <= 0: nu_0 = nu0_scale |J g|^2 / |g|^2 at u, as at the start of og_lm):
 * the step s = P(u + delta) - u of Eq. (9) (P: projection onto the constraint set), its
 * model decrease, the actual decrease, rho of Eq. (12), the acceptance rho > eta and the
 * next damping (before clamping).
 * u is not changed: this is the "s_k = LMA(u_k)" of Alg. 2, whose caller decides. */
int og_lm_trial(const og_geom* gin, const og_params* pr, const double* y, const double* lam,
                const double* mu, double nu, double* s, og_trial* out) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    const og_geom* g = &o.g;
    int n = g->n, np = n * n, m = g->n_angles * g->n_det;
    memset(out, 0, sizeof *out);
    double* r = malloc(sizeof(double) * m);
    double* rt = malloc(sizeof(double) * m);
    double* Js = malloc(sizeof(double) * m);
    double* Wl = malloc(sizeof(double) * np);
    double* Wm = malloc(sizeof(double) * np);
    double* grad = malloc(sizeof(double) * 2 * np);
    double* rhs = malloc(sizeof(double) * 2 * np);
    double* delta = malloc(sizeof(double) * 2 * np);
    double* ut = malloc(sizeof(double) * 2 * np);
    double* tmp = malloc(sizeof(double) * np);
    double f = og_objective(g, pr, lam, mu, y, r);
    og_reg_weights(n, pr->tv_eps, lam, Wl);
    og_reg_weights(n, pr->tv_eps, mu, Wm);
    og_gradient(g, pr, lam, mu, r, Wl, Wm, grad, tmp);
    if (!(nu > 0.0)) {
        double gg = og_dot(2 * np, grad, grad);
        nu = 1.0;
        if (gg > 0.0) {
            og_jvp(g, lam, mu, grad, grad + np, Js);
            nu = pr->nu0_scale * og_dot(m, Js, Js) / gg;
        }
        if (!(nu > 0.0)) nu = 1.0;
        out->nu0 = nu;
    }
    if (pr->inner_solver == 1) {
        out->cg_iters = og_sgp(g, pr, lam, mu, Wl, Wm, nu, grad, delta);
    } else {
        for (int i = 0; i < 2 * np; ++i) rhs[i] = -grad[i];
        out->cg_iters = og_cg(g, pr, lam, mu, Wl, Wm, nu, rhs, delta);
    }
    for (int i = 0; i < np; ++i) {
        ut[i] = lam[i] + delta[i];
        ut[np + i] = mu[i] + delta[np + i];
        og_project_px(pr, &ut[i], &ut[np + i]);
        s[i] = ut[i] - lam[i];
        s[np + i] = ut[np + i] - mu[i];
    }
    double pred = og_model_decrease(g, pr, lam, mu, grad, Wl, Wm, s, Js, tmp);
    double ft = og_objective(g, pr, ut, ut + np, y, rt);
    double ared = f - ft;
    double rho = (pred > 0.0 && isfinite(ft)) ? ared / pred : -INFINITY;
    out->f = f;
    out->pred = pred;
    out->ared = ared;
    out->rho = rho;
    out->accept = rho > pr->eta;
    out->nu_next = rho < pr->rho_lo ? nu * pr->nu_up : (rho > pr->rho_hi ? nu * pr->nu_down : nu);
    free(r);
    free(rt);
    free(Js);
    free(Wl);
    free(Wm);
    free(grad);
    free(rhs);
    free(delta);
    free(ut);
    free(tmp);
    return 0;
}

/* The convergence check of Prop. conv_check / Alg. 2 for a proposal u~ = (pl, pm) made
 * at the feasible point u with the LM step s_k: with s~ = P(u~) - u (the proposal
 * projected onto the constraint set, as the LM step is),
 *   accept u~ iff rho(s~) > eta and m_k(s~) <= m_k(s_k),
 * m_k(s~) <= m_k(s_k) being m_k(0) - m_k(s~) >= m_k(0) - m_k(s_k); rho as in Eq. (12)
 * (-inf when the model predicts no decrease). */
int og_check_proposal(const og_geom* gin, const og_params* pr, const double* y, const double* lam,
                      const double* mu, const double* s_step, const double* pl, const double* pm,
                      og_check* out) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    const og_geom* g = &o.g;
    int n = g->n, np = n * n, m = g->n_angles * g->n_det;
    memset(out, 0, sizeof *out);
    double* r = malloc(sizeof(double) * m);
    double* rt = malloc(sizeof(double) * m);
    double* Js = malloc(sizeof(double) * m);
    double* Wl = malloc(sizeof(double) * np);
    double* Wm = malloc(sizeof(double) * np);
    double* grad = malloc(sizeof(double) * 2 * np);
    double* ut = malloc(sizeof(double) * 2 * np);
    double* sp = malloc(sizeof(double) * 2 * np);
    double* tmp = malloc(sizeof(double) * np);
    double f = og_objective(g, pr, lam, mu, y, r);
    og_reg_weights(n, pr->tv_eps, lam, Wl);
    og_reg_weights(n, pr->tv_eps, mu, Wm);
    og_gradient(g, pr, lam, mu, r, Wl, Wm, grad, tmp);
    for (int i = 0; i < np; ++i) {
        ut[i] = pl[i];
        ut[np + i] = pm[i];
        og_project_px(pr, &ut[i], &ut[np + i]);
        sp[i] = ut[i] - lam[i];
        sp[np + i] = ut[np + i] - mu[i];
    }
    double pred_s = og_model_decrease(g, pr, lam, mu, grad, Wl, Wm, s_step, Js, tmp);
    double pred_p = og_model_decrease(g, pr, lam, mu, grad, Wl, Wm, sp, Js, tmp);
    double fp = og_objective(g, pr, ut, ut + np, y, rt);
    double ared = f - fp;
    double rho = (pred_p > 0.0 && isfinite(fp)) ? ared / pred_p : -INFINITY;
    out->f = f;
    out->pred_step = pred_s;
    out->pred_prop = pred_p;
    out->ared_prop = ared;
    out->rho_prop = rho;
    out->accept = rho > pr->eta && pred_p >= pred_s;
    free(r);
    free(rt);
    free(Js);
    free(Wl);
    free(Wm);
    free(grad);
    free(ut);
    free(sp);
    free(tmp);
    return 0;
}

/* Initial guess (the paper does not state one): mu = mu_init everywhere (the known
 * water value), lambda = c everywhere with c = sum y / sum A(1, mu_init) so that the
 * total counts match, both projected onto the box. */
int og_initial_guess(const og_geom* gin, const double* y, double mu_init, double lambda_max,
                     double mu_max, double* lam, double* mu) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    int np = o.g.n * o.g.n, m = o.g.n_angles * o.g.n_det;
    double* ones = malloc(sizeof(double) * np);
    double* ya = malloc(sizeof(double) * m);
    for (int i = 0; i < np; ++i) {
        ones[i] = 1.0;
        mu[i] = og_clamp(mu_init, 0.0, mu_max);
    }
    og_forward(&o.g, ones, mu, ya);
    double sy = 0.0, sa = 0.0;
    for (int i = 0; i < m; ++i) {
        sy += y[i];
        sa += ya[i];
    }
    double cst = sa > 0.0 ? sy / sa : 0.0;
    for (int i = 0; i < np; ++i) lam[i] = og_clamp(cst, 0.0, lambda_max);
    free(ones);
    free(ya);
    return 0;
}

/* Geometry helpers exposed for tests: samples per ray, detector pitch, fov radius. */
int og_geom_info(const og_geom* gin, int32_t* T, double* pitch, double* radius, int32_t* n_banks) {
    og_ctx o;
    if (og_setup(gin, &o)) return 1;
    *T = o.T;
    *pitch = o.p;
    *radius = o.r;
    *n_banks = o.g.n_banks;
    return 0;
}

int og_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops (the angle loops of og_forward, og_jvp and og_vjp); n <= 0
 * restores the default.  Only the timing of the oracle changes, never a result: every
 * reduction over angles is summed in a fixed order of chunks (og_set_vjp_chunks). */
void og_set_num_threads(int n) {
#ifdef _OPENMP
    static int dflt = 0;
    if (dflt == 0) dflt = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : dflt);
#else
    (void)n;
#endif
}

/* The parameters of LM iteration k under the continuation of Sec. 3.1 (og_params_at). */
void og_params_at_k(const og_params* pr, int k, og_params* out) { *out = og_params_at(pr, k); }
