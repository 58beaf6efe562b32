// kernels.cuh -- device helpers and kernel launch interfaces of the CUDA library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <vector>

#include "pget_internal.cuh"

namespace pget {

// host-side count of kernel launches made by the library (diagnostics)
void note_launch(int k = 1);
long long launch_count();

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ float exp2_(float x) { return exp2f(x); }
__device__ __forceinline__ double exp2_(double x) { return exp2(x); }

// w00 a00 + w10 a10 + w01 a01 + w11 a11 on (lambda, mu) pairs; packed FP32x2 on float
__device__ __forceinline__ float2 bilerp2(float w00, float w10, float w01, float w11, float2 a00, float2 a10,
                                          float2 a01, float2 a11) {
    float2 r = __fmul2_rn(make_float2(w00, w00), a00);
    r = __ffma2_rn(make_float2(w10, w10), a10, r);
    r = __ffma2_rn(make_float2(w01, w01), a01, r);
    return __ffma2_rn(make_float2(w11, w11), a11, r);
}
__device__ __forceinline__ double2 bilerp2(double w00, double w10, double w01, double w11, double2 a00,
                                           double2 a10, double2 a01, double2 a11) {
    return make_double2(w00 * a00.x + w10 * a10.x + w01 * a01.x + w11 * a11.x,
                        w00 * a00.y + w10 * a10.y + w01 * a01.y + w11 * a11.y);
}
// t + w g on pairs
__device__ __forceinline__ float2 fma2(float w, float2 g, float2 t) { return __ffma2_rn(make_float2(w, w), g, t); }
__device__ __forceinline__ double2 fma2(double w, double2 g, double2 t) {
    return make_double2(t.x + w * g.x, t.y + w * g.y);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Running sum along a ray; KAHAN selects compensated summation (the compensation holds
// the rounding excess of the last addition, the value is s - c).
template <typename T, bool KAHAN> struct Acc {
    T s, c;
    __device__ __forceinline__ void init() { s = T(0); c = T(0); }
    __device__ __forceinline__ void add(T x) {
        if constexpr (KAHAN) {
            T y = x - c;
            T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ T val() const {
        if constexpr (KAHAN) return s - c;
        else return s;
    }
};

// Sample position along one ray in the canonical frame of its view.
//   float paths: 32.32 fixed point, exact steps (no drift along a ray);
//   double path: X = X0 + j dX evaluated per sample.
template <typename T> struct Pos;

template <> struct Pos<float> {
    long long X, Y, dX, dY;
    __device__ __forceinline__ void init(const ViewDev& v, int i, int j) {
        X = v.X00 + (long long)i * v.dXr + (long long)j * v.dXs;
        Y = v.Y00 + (long long)i * v.dYr + (long long)j * v.dYs;
        dX = v.dXs;
        dY = v.dYs;
    }
    __device__ __forceinline__ void back() {
        X -= dX;
        Y -= dY;
    }
    __device__ __forceinline__ int ix() const { return (int)(X >> 32); }
    __device__ __forceinline__ int iy() const { return (int)(Y >> 32); }
    __device__ __forceinline__ float ax() const {
        return __uint2float_rn((unsigned)(X & 0xffffffffull)) * 2.3283064365386963e-10f;
    }
    __device__ __forceinline__ float ay() const {
        return __uint2float_rn((unsigned)(Y & 0xffffffffull)) * 2.3283064365386963e-10f;
    }
    __device__ __forceinline__ float yf() const { return __ll2float_rn(Y) * 2.3283064365386963e-10f; }
};

template <> struct Pos<double> {
    double X0, Y0, dX, dY, X, Y, fx, fy;
    int j;
    __device__ __forceinline__ void eval() {
        X = fma((double)j, dX, X0);
        Y = fma((double)j, dY, Y0);
        fx = floor(X);
        fy = floor(Y);
    }
    __device__ __forceinline__ void init(const ViewDev& v, int i, int j_) {
        X0 = fma((double)i, v.dXrd, v.X00d);  // explicit fma: the host repeats it exactly
        Y0 = fma((double)i, v.dYrd, v.Y00d);
        dX = v.dXsd;
        dY = v.dYsd;
        j = j_;
        eval();
    }
    __device__ __forceinline__ void back() {
        --j;
        eval();
    }
    __device__ __forceinline__ int ix() const { return (int)fx; }
    __device__ __forceinline__ int iy() const { return (int)fy; }
    __device__ __forceinline__ double ax() const { return X - fx; }
    __device__ __forceinline__ double ay() const { return Y - fy; }
    __device__ __forceinline__ float yf() const { return (float)Y; }
};

// kVjpP is the adjoint with phase-coloured row buffers; callers ask for kVjp and the
// launch takes kVjpP when the adjoint's plan has phases (WalkPlan::nph > 0)
enum WalkMode { kFwd = 0, kJvp = 1, kVjp = 2, kVjpP = 3 };

struct WalkArgs {
    const ViewDev* views;
    int n, T, P, Yc, nchunks, sb_cap;
    int Ps;                    // shared-memory row pitch of a staged chunk (elements)
    int nst;                   // VJP: stride between stencil planes (>= threads)
    int nph, Pb, phs;          // kVjpP: phases, row pitch and phase stride of the row buffers (elements)
    double h;
    const void* u_img[2];      // padded interleaved (lambda, mu): [0] normal, [1] transposed
    const void* p_img[2];      // JVP: padded interleaved (dlambda, dmu)
    void* slot_val;            // FWD: per-slot ray total out (optional); VJP: in
    int max_slots, n_det, n_banks, nb, n_sub;
    const int* det_slot;       // [n_det][n_sub]
    const void* w;             // [n_sub] sub-ray weights (element type of the path)
    const int2* clip;          // [n_views * max_slots] conservative sample range per ray
    void* y_out;               // FWD / JVP: [n_angles][n_det]
    const void* r_in;          // VJP: [n_angles][n_det]
    const int* src_off;
    const int* src_det;
    const void* src_w;         // weights of the sub-rays on each slot (element type of the path)
    void* gpart;               // VJP: [n_views][2][n][n], pre-flip canonical layout
    const int2* win;           // VJP: [n_views][nchunks] (first slot, count) of the rays with
                               //      samples in the chunk; stencil column = slot - first
    const int* group_off;      // VJP: CTA g handles views group_view[group_off[g] .. group_off[g+1])
    const int* group_view;     //      (null: CTA g handles view g)
    const int* cta_order;      // CTA b takes view (FWD / JVP) or view group (VJP) cta_order[b]:
                               //      longest rays first, so that the last wave holds the
                               //      shortest (null: b)
    const void* depth;         // [T] (w_j, c_j) pairs (element type of the path): depth factors
                               //      of Eq. (5); null without tables
    const int* stop;           // optional: skip the launch when *stop != 0
    long long wait_ns;         // limit of one chunk-copy wait (0: 1 s)
    int tx_extra;              // test aid: bytes added to the first chunk's expected copy
                               // size, so that its wait runs out (0 in normal use)
    int* err;                  // error flags (bit 1: adjoint stencil bound, bit 2: chunk copy wait timed out)
    // batched launches (grid.y = n_items independent items of one geometry): byte strides
    // between the items' packed layouts (u_img and p_img), sinograms (y_out and r_in), ray
    // totals (slot_val) and adjoint partial images (gpart); n_items 0 or 1 and strides 0
    // for one item
    int n_items;
    long long s_img, s_sino, s_slot, s_part;
};

struct WalkPlan {
    int threads = 0, Yc = 0, nchunks = 0, sb_cap = 0, Ps = 0, nst = 0;
    int nph = 0, Pb = 0, phs = 0;  // adjoint with phase-coloured row buffers (nph > 0)
    size_t smem = 0;
    std::vector<int2> win;  // VJP: [view][chunk] ray window of each chunk
};

// Rows of the first (largest j) and last valid sample of every ray, computed with the
// kernels' own arithmetic (32.32 fixed point, or double fma); (INT_MIN, INT_MIN) for a
// ray without valid samples.  [view][max_slots].
void ray_rows(const Geometry& g, bool f64, std::vector<int2>* rows);

// h log2(e): the packed images hold mu in units where the attenuation sum is a power of 2
inline double attenuation_scale(const Geometry& g) { return g.h * 1.4426950408889634; }

// Phases the adjoint's row buffers need for this geometry's slot lattice (0: a degenerate
// lattice); see the derivation in walk.cu.
int adjoint_phases_needed(const Geometry& g);

// Plan (threads, rows per chunk, shared memory) for one walk mode.
// The adjoint plan needs the ray rows (ray_rows) to size its stencil windows.
WalkPlan plan_walk(const Geometry& g, int P, int mode, bool f64, size_t smem_budget,
                   const std::vector<int2>* rows = nullptr);

// Permit the planned dynamic shared memory (call before capturing a graph).
cudaError_t prepare_walk(int mode, int precision, const WalkPlan& plan);

// Resident CTAs per SM of a planned walk kernel.
int walk_occupancy(int mode, int precision, const WalkPlan& plan);

// Launch one walk kernel over all views of the geometry.
cudaError_t launch_walk(int mode, int precision, const WalkPlan& plan, const WalkArgs& a,
                        int n_views, cudaStream_t st);

}  // namespace pget
