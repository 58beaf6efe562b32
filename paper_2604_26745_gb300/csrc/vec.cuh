// vec.cuh -- launch interfaces of vec.cu and the device-resident solver state.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "kernels.cuh"

namespace pget {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs; fixed so reductions are deterministic

// CG state; the gradient-projection solver reuses it: rr = |unit-step projected gradient|,
// bnorm = its first value (< 0 before), pq = <grad q, d>, dd = |d|^2, alpha = step length,
// beta = line-search step, iters and stop as for CG
struct CgState {
    double rr, pq, alpha, beta, bnorm, tol, dd;
    double rr_prev;  // CG: |res|^2 of the previous step (the fused direction update divides by it)
    int iters, stop;
};

// Constraint set of one pixel's pair (lambda, mu), Sec. 2.2: the box [0, lmax] x [0, mmax]
// and, when lin is set, the linear bound lambda <= k mu + b (k, b >= 0).  t_hi is the
// largest mu of the bound's segment inside the box, den = k^2 + 1.
struct Feas {
    double lmax, mmax, k, b, t_hi, den;
    int lin;
};
inline Feas make_feas(double lmax, double mmax, int lin, double k, double b) {
    Feas f{lmax, mmax, k, b, mmax, k * k + 1.0, lin};
    if (k > 0.0 && (lmax - b) / k < f.t_hi) f.t_hi = (lmax - b) / k;
    return f;
}

struct LmState {
    double f, f0, nu, nu0;
    double sg, sHs, JsJs, rtrt, Rl, Rm, gg;
    double init_sa, init_sy;         // initial guess: sum A(1, mu0) and sum y
    int accept, no_grad, iter, accepted, cg_total, pad;
    CgState cg;
    double tr_f[PGET_TRACE], tr_rho[PGET_TRACE], tr_nu[PGET_TRACE], tr_pred[PGET_TRACE], tr_ared[PGET_TRACE];
    int tr_acc[PGET_TRACE], tr_cg[PGET_TRACE];
};

struct LmParamsDev {
    double eta, rho_lo, rho_hi, nu_up, nu_down, nu_min, nu_max;
};

template <typename T> struct RedArgs {
    int groups = 0;
    int n = 0;
    T* out = nullptr;            // [2][n][n]
    const T* v = nullptr;        // optional: add alpha grad^T W grad v + nu v
    const T* Wl = nullptr;
    const T* Wm = nullptr;
    double alpha_l = 0, alpha_m = 0;
    double nu = 0;
    const double* nu_dev = nullptr;  // if set, nu is read from the device
    const T* dotv = nullptr;     // optional: per-block partials of <dotv, out>
    double* part = nullptr;
    const int* skip = nullptr;
    // optional geometry priors (Eq. (6)): adds 2 geo (1 - M)^2 (v - c) with the mask M,
    // weights geo_l / geo_m and c = geo_cm on the mu field when geo_offset (gradient), else 0
    const T* gmask = nullptr;
    double geo_l = 0, geo_m = 0, geo_cm = 0;
    int geo_offset = 0;
};

// planar (lambda, mu) of the solver's type TV -> the padded interleaved layouts of the ray
// kernels' type TW
template <typename TV, typename TW>
void pack(const TV* lam, const TV* mu, int n, int P, double mu_scale, void* out_n, void* out_t, const int* skip,
          cudaStream_t st);
// dst[i] = src[i] (sinograms between the solver's and the ray kernels' types)
template <typename A, typename B>
void convert(const A* src, B* dst, size_t m, const int* skip, cudaStream_t st);
template <typename T>
void reg_weights(const T* u, int n, double eps, T* W, const int* skip, cudaStream_t st);
template <typename T>
void reg_apply(const T* v, const T* W, int n, double alpha, T* out, cudaStream_t st);
// alpha * R(u) (smoothed TV or quadratic), plus galpha |(1 - M)(u - gc)|^2 when gmask is set
template <typename T>
void reg_value(const T* u, int n, double alpha, double eps, double* part, const int* skip, cudaStream_t st,
               const T* gmask = nullptr, double galpha = 0.0, double gc = 0.0);
template <typename T>
void dot(const T* a, const T* b, size_t m, double* part, const int* skip, cudaStream_t st);
void finish_sum(const double* part, double* dst, const int* skip, cudaStream_t st);
// adjoint view reduction: partial images of the ray kernels' type TP, result and the fused
// prior / damping / dot of the solver's type T
template <typename T, typename TP>
void reduce_views(const TP* gpart, int n, int n_views, int n0, int groups, TP* part2, const RedArgs<T>& ra,
                  bool kahan, cudaStream_t st);
template <typename T>
void sub_dot(const T* a, const T* b, T* out, size_t m, double* part, const int* skip, cudaStream_t st);
// projection onto the constraint set, in place: stacked [lambda; mu] / separate images
template <typename T>
void project_set(T* u, size_t nn, const Feas& f, cudaStream_t st);
template <typename T>
void project_pair(T* lam, T* mu, size_t nn, const Feas& f, cudaStream_t st);
template <typename T>
void fill(T* u, size_t m, double v, cudaStream_t st);
template <typename T>
void cg_init(const T* b, T* x, T* res, T* p, size_t m, double scale_b, double tol, double* part, CgState* cg,
             cudaStream_t st);
// fused CG step (finish of <p, q>, x and res update, partials of |res|^2 into part_rr) and
// direction update (finish of |res|^2, p update, packing of p for the next JVP)
template <typename T>
void cg_step(T* x, T* res, const T* p, const T* q, size_t m, const double* part_pq, double* part_rr, CgState* cg,
             cudaStream_t st);
template <typename T, typename TW>
void cg_dir_pack(T* p, const T* res, const double* part_rr, CgState* cg, int n, int P, double mu_scale, void* out_n,
                 void* out_t, cudaStream_t st);
template <typename T>
void lm_step(const T* u, const T* x, T* ut, T* s, size_t nn, const Feas& f, cudaStream_t st);
template <typename T>
void lm_model(const T* s, const T* g, const T* Wl, const T* Wm, int n, double al, double am, double* pa,
              double* pb, cudaStream_t st, const T* gmask = nullptr, double geo_l = 0.0, double geo_m = 0.0);
void lm_decide(LmState* L, const LmParamsDev& P, cudaStream_t st);
void lm_init_f(LmState* L, double nu0_scale, cudaStream_t st);
// gradient projection on the constrained LM subproblem (see vec.cu)
template <typename T>
void sgp_init(const T* g, T* gq, T* x, size_t m, double tol, CgState* cg, cudaStream_t st);
template <typename T>
void sgp_dir(const T* u, const T* x, const T* gq, T* d, size_t nn, const Feas& f, double* p_pg,
             double* p_gd, double* p_dd, CgState* cg, cudaStream_t st);
void sgp_step(const double* p_dAd, const double* p_AdAd, CgState* cg, cudaStream_t st);
template <typename T>
void sgp_update(T* x, T* gq, const T* d, const T* Ad, size_t m, const CgState* cg, cudaStream_t st);
void lm_refresh_f(LmState* L, cudaStream_t st);
template <typename T>
void copy_if(T* dst, const T* src, size_t m, const int* flag, cudaStream_t st);
template <typename T>
void scale(T* y, size_t m, double c, cudaStream_t st);
// u[i] = clamp(*num / *den, 0, hi) (0 when *den <= 0), for i < m
template <typename T>
void fill_ratio(T* u, size_t m, const double* num, const double* den, double hi, cudaStream_t st);

}  // namespace pget
