// vec.cu -- image packing, the view reduction of the VJP, the prior (smoothed TV), the
// FP64 dot products and the CG / trust-region vector and scalar steps.
//
// Vectors u = (lambda, mu) are planar [2][n][n] (lambda block, then mu block).  Dot
// products accumulate in double per thread, per block (fixed tree) and over blocks in
// block order (finish kernels), so every result is deterministic.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "kernels.cuh"
#include "vec.cuh"

namespace pget {

// ------------------------------------------------------------------------ packing
// planar lambda, mu -> padded interleaved images, normal ([iy+1][ix+1]) and transposed
// ([ix+1][iy+1]); the one-pixel border stays zero (bilinear samples see zero outside).
// The second component is stored as mu * mu_scale (the ray kernels take h log2(e), so
// the attenuation sum is directly the exponent of 2).
template <typename TV, typename TW>
__global__ void pack_kernel(const TV* __restrict__ lam, const TV* __restrict__ mu, int n, int P, TV mu_scale,
                            typename Vec2<TW>::type* __restrict__ out_n,
                            typename Vec2<TW>::type* __restrict__ out_t, const int* skip) {
    using T2 = typename Vec2<TW>::type;
    if (skip && *skip) return;
    __shared__ T2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int iy = by + k, ix = bx + threadIdx.x;
        if (iy < n && ix < n) {
            T2 v = mk2((TW)lam[(size_t)iy * n + ix], (TW)(mu_scale * mu[(size_t)iy * n + ix]));
            out_n[(size_t)(iy + 1) * P + ix + 1] = v;
            tile[k][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int ix = bx + k, iy = by + threadIdx.x;
        if (iy < n && ix < n) out_t[(size_t)(ix + 1) * P + iy + 1] = tile[threadIdx.x][k];
    }
}

template <typename TV, typename TW>
void pack(const TV* lam, const TV* mu, int n, int P, double mu_scale, void* out_n, void* out_t, const int* skip,
          cudaStream_t st) {
    dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
    pack_kernel<TV, TW><<<grid, block, 0, st>>>(lam, mu, n, P, (TV)mu_scale, (typename Vec2<TW>::type*)out_n,
                                                (typename Vec2<TW>::type*)out_t, skip);
    note_launch();
}
template void pack<float, float>(const float*, const float*, int, int, double, void*, void*, const int*, cudaStream_t);
template void pack<double, double>(const double*, const double*, int, int, double, void*, void*, const int*,
                                   cudaStream_t);
template void pack<double, float>(const double*, const double*, int, int, double, void*, void*, const int*,
                                  cudaStream_t);

// dst = src element by element (sinograms between the solver's and the ray kernels' types)
template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ src, B* __restrict__ dst, size_t m, const int* skip) {
    if (skip && *skip) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}
template <typename A, typename B>
void convert(const A* src, B* dst, size_t m, const int* skip, cudaStream_t st) {
    convert_kernel<A, B><<<kRedBlocks, 256, 0, st>>>(src, dst, m, skip);
    note_launch();
}
template void convert<float, double>(const float*, double*, size_t, const int*, cudaStream_t);
template void convert<double, float>(const double*, float*, size_t, const int*, cudaStream_t);

// ------------------------------------------------------------------------ prior
// forward differences with a zero-flux border; W = 1/sqrt(|grad u|^2 + eps^2) or 1
template <typename T>
__device__ __forceinline__ void grad_at(const T* u, int n, int ix, int iy, T* gx, T* gy) {
    const size_t i = (size_t)iy * n + ix;
    *gx = ix < n - 1 ? u[i + 1] - u[i] : T(0);
    *gy = iy < n - 1 ? u[i + n] - u[i] : T(0);
}

// alpha grad^T diag(W) grad v at pixel (ix, iy)
template <typename T>
__device__ __forceinline__ T reg_at(const T* v, const T* W, T alpha, int n, int ix, int iy) {
    const size_t i = (size_t)iy * n + ix;
    T gx, gy, acc = T(0);
    grad_at(v, n, ix, iy, &gx, &gy);
    acc -= W[i] * gx + W[i] * gy;
    if (ix > 0) {
        T gxl, gyl;
        grad_at(v, n, ix - 1, iy, &gxl, &gyl);
        acc += W[i - 1] * gxl;
    }
    if (iy > 0) {
        T gxd, gyd;
        grad_at(v, n, ix, iy - 1, &gxd, &gyd);
        acc += W[i - n] * gyd;
    }
    return alpha * acc;
}

template <typename T>
__global__ void reg_weights_kernel(const T* __restrict__ u, int n, double eps, T* __restrict__ W,
                                   const int* skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * n) return;
    const int iy = i / n, ix = i - iy * n;
    T gx, gy;
    grad_at(u, n, ix, iy, &gx, &gy);
    W[i] = eps > 0 ? T(1) / sqrt(gx * gx + gy * gy + (T)(eps * eps)) : T(1);
}

template <typename T>
void reg_weights(const T* u, int n, double eps, T* W, const int* skip, cudaStream_t st) {
    int tot = n * n;
    reg_weights_kernel<T><<<(tot + 255) / 256, 256, 0, st>>>(u, n, eps, W, skip);
    note_launch();
}
template void reg_weights<float>(const float*, int, double, float*, const int*, cudaStream_t);
template void reg_weights<double>(const double*, int, double, double*, const int*, cudaStream_t);

template <typename T>
__global__ void reg_apply_kernel(const T* __restrict__ v, const T* __restrict__ W, int n, double alpha,
                                 T* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * n) return;
    const int iy = i / n, ix = i - iy * n;
    out[i] = reg_at(v, W, (T)alpha, n, ix, iy);
}

template <typename T>
void reg_apply(const T* v, const T* W, int n, double alpha, T* out, cudaStream_t st) {
    int tot = n * n;
    reg_apply_kernel<T><<<(tot + 255) / 256, 256, 0, st>>>(v, W, n, alpha, out);
    note_launch();
}
template void reg_apply<float>(const float*, const float*, int, double, float*, cudaStream_t);
template void reg_apply<double>(const double*, const double*, int, double, double*, cudaStream_t);

// ------------------------------------------------------------------ block reduction
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) r += red[w];
    return r;  // valid in thread 0
}

// R(u) = alpha sum sqrt(|grad u|^2 + eps^2)  or  alpha/2 sum |grad u|^2 ; per-block partials
template <typename T>
__global__ void reg_value_kernel(const T* __restrict__ u, int n, double alpha, double eps,
                                 double* __restrict__ part, const int* skip, const T* __restrict__ gmask,
                                 double galpha, double gc) {
    if (skip && *skip) return;
    double acc = 0.0, gacc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
        const int iy = i / n, ix = i - iy * n;
        T gx, gy;
        grad_at(u, n, ix, iy, &gx, &gy);
        double s2 = (double)gx * gx + (double)gy * gy;
        acc += eps > 0 ? sqrt(s2 + eps * eps) : 0.5 * s2;
        if (gmask) {  // geometry prior of Eq. (6)
            const double pv = (1.0 - (double)gmask[i]) * ((double)u[i] - gc);
            gacc += pv * pv;
        }
    }
    double s = alpha * block_sum(acc);
    if (gmask) s += galpha * block_sum(gacc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
void reg_value(const T* u, int n, double alpha, double eps, double* part, const int* skip,
               cudaStream_t st, const T* gmask, double galpha, double gc) {
    reg_value_kernel<T><<<kRedBlocks, 256, 0, st>>>(u, n, alpha, eps, part, skip, gmask, galpha, gc);
    note_launch();
}
template void reg_value<float>(const float*, int, double, double, double*, const int*, cudaStream_t,
                               const float*, double, double);
template void reg_value<double>(const double*, int, double, double, double*, const int*, cudaStream_t,
                                const double*, double, double);

// ------------------------------------------------------------------------ dots
template <typename T>
__global__ void dot_kernel(const T* __restrict__ a, const T* __restrict__ b, size_t m,
                           double* __restrict__ part, const int* skip) {
    if (skip && *skip) return;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
void dot(const T* a, const T* b, size_t m, double* part, const int* skip, cudaStream_t st) {
    dot_kernel<T><<<kRedBlocks, 256, 0, st>>>(a, b, m, part, skip);
    note_launch();
}
template void dot<float>(const float*, const float*, size_t, double*, const int*, cudaStream_t);
template void dot<double>(const double*, const double*, size_t, double*, const int*, cudaStream_t);

// Sum of the kRedBlocks partials by one warp in a fixed order (lane l adds partials
// l, l+32, ...; then a fixed shuffle tree): deterministic, and the loads overlap.
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ part) {
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += 32) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;  // the same value in every lane
}

// sum kRedBlocks partials into *dst
__global__ void finish_sum_kernel(const double* __restrict__ part, double* dst, const int* skip) {
    if (skip && *skip) return;
    const double s = warp_sum_partials(part);
    if (threadIdx.x == 0) *dst = s;
}
void finish_sum(const double* part, double* dst, const int* skip, cudaStream_t st) {
    finish_sum_kernel<<<1, 32, 0, st>>>(part, dst, skip);
    note_launch();
}

// ---------------------------------------------------------------- view reduction
// Stage 1: block (tile, view group) sums the partial images of its views over a 32 x 32
// pixel tile.  The partial images come sorted by orientation: views [0, n0) wrote the
// normal frame, views [n0, n_views) the transposed one ([ix][iy]).  Groups [0, g0) split
// the first range, groups [g0, groups) the second, so every block sums one orientation
// with no per-view test (its loads stay independent across the unrolled views); a
// transposed block turns its tile once through shared memory.
// (float: at most 64 registers, so that four 256-thread blocks fit an SM and the
// tiles x groups grid of about 2 x 304 blocks runs in a single wave)
template <typename T, bool KAHAN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 && !KAHAN ? 4 : 3)
    reduce_views_kernel(const T* __restrict__ gpart, int n, int n_views, int n0, int groups, int g0,
                        T* __restrict__ out2, const int* skip) {
    using T2 = typename Vec2<T>::type;
    if (skip && *skip) return;
    __shared__ T2 tile[32][33];
    const int tiles_x = (n + 31) / 32;
    const int tl = blockIdx.x % (tiles_x * tiles_x), grp = blockIdx.x / (tiles_x * tiles_x);
    const int bx = (tl % tiles_x) * 32, by = (tl / tiles_x) * 32;
    const bool tr = grp >= g0;
    const int c0 = tr ? n0 : 0, cn = tr ? n_views - n0 : n0;
    const int gi = tr ? grp - g0 : grp, gn = tr ? groups - g0 : g0;
    const int v0 = c0 + (int)((long long)cn * gi / gn), v1 = c0 + (int)((long long)cn * (gi + 1) / gn);
    const size_t nn = (size_t)n * n;
    Acc<T, KAHAN> a[2][4];
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < 4; ++k) a[f][k].init();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int rb = tr ? bx : by, cb = tr ? by : bx;  // stored rows and columns of the tile
    constexpr int kUnroll = sizeof(T) == 4 && !KAHAN ? 4 : 2;  // loads in flight within 64 registers
#pragma unroll kUnroll
    for (int v = v0; v < v1; ++v) {
        const T* gp = gpart + (size_t)v * 2 * nn;
        for (int k = 0; k < 4; ++k) {
            const int r = rb + ty + 8 * k, c = cb + tx;
            if (r < n && c < n) {
                a[0][k].add(gp[(size_t)r * n + c]);
                a[1][k].add(gp[nn + (size_t)r * n + c]);
            }
        }
    }
    T* o = out2 + (size_t)grp * 2 * nn;
    if (tr) {  // uniform per block
        for (int k = 0; k < 4; ++k) tile[ty + 8 * k][tx] = mk2(a[0][k].val(), a[1][k].val());
        __syncthreads();
        for (int k = 0; k < 4; ++k) {
            const int iy = by + ty + 8 * k, ix = bx + tx;
            if (iy < n && ix < n) {
                const T2 tv = tile[tx][ty + 8 * k];
                o[(size_t)iy * n + ix] = tv.x;
                o[nn + (size_t)iy * n + ix] = tv.y;
            }
        }
    } else {
        for (int k = 0; k < 4; ++k) {
            const int iy = by + ty + 8 * k, ix = bx + tx;
            if (iy < n && ix < n) {
                o[(size_t)iy * n + ix] = a[0][k].val();
                o[nn + (size_t)iy * n + ix] = a[1][k].val();
            }
        }
    }
}

// Stage 1 for float images with n divisible by 4: as reduce_views_kernel, but every thread
// sums one row segment of four pixels (16-byte loads and stores; the views in the same
// order, so the sums are the same).
template <bool KAHAN>
__global__ void __launch_bounds__(256, KAHAN ? 3 : 4)
    reduce_views4_kernel(const float* __restrict__ gpart, int n, int n_views, int n0, int groups, int g0,
                         float* __restrict__ out2, const int* skip) {
    if (skip && *skip) return;
    __shared__ float2 tile[32][33];
    const int tiles_x = (n + 31) / 32;
    const int tl = blockIdx.x % (tiles_x * tiles_x), grp = blockIdx.x / (tiles_x * tiles_x);
    const int bx = (tl % tiles_x) * 32, by = (tl / tiles_x) * 32;
    const bool tr = grp >= g0;
    const int c0 = tr ? n0 : 0, cn = tr ? n_views - n0 : n0;
    const int gi = tr ? grp - g0 : grp, gn = tr ? groups - g0 : g0;
    const int v0 = c0 + (int)((long long)cn * gi / gn), v1 = c0 + (int)((long long)cn * (gi + 1) / gn);
    const size_t nn = (size_t)n * n;
    const int t = threadIdx.y * 32 + threadIdx.x;
    const int rr = t >> 3, cc = (t & 7) * 4;         // tile row, first of its four columns
    const int r = (tr ? bx : by) + rr, c = (tr ? by : bx) + cc;  // stored row and column
    Acc<float, KAHAN> a[2][4];
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < 4; ++k) a[f][k].init();
    if (r < n && c < n) {  // c and n are multiples of 4: the segment lies inside the row
        const size_t off = (size_t)r * n + c;
#pragma unroll 4
        for (int v = v0; v < v1; ++v) {
            const float* gp = gpart + (size_t)v * 2 * nn + off;
            const float4 x = *reinterpret_cast<const float4*>(gp);
            const float4 y = *reinterpret_cast<const float4*>(gp + nn);
            a[0][0].add(x.x);
            a[0][1].add(x.y);
            a[0][2].add(x.z);
            a[0][3].add(x.w);
            a[1][0].add(y.x);
            a[1][1].add(y.y);
            a[1][2].add(y.z);
            a[1][3].add(y.w);
        }
    }
    float* o = out2 + (size_t)grp * 2 * nn;
    if (tr) {  // stored [ix][iy]: the thread holds ix = r, iy = c + k; turn the tile (uniform per block)
        for (int k = 0; k < 4; ++k) tile[cc + k][rr] = make_float2(a[0][k].val(), a[1][k].val());
        __syncthreads();
        const int iy = by + rr, ix = bx + cc;
        if (iy < n && ix < n) {
            const float2 e0 = tile[rr][cc], e1 = tile[rr][cc + 1], e2 = tile[rr][cc + 2], e3 = tile[rr][cc + 3];
            *reinterpret_cast<float4*>(o + (size_t)iy * n + ix) = make_float4(e0.x, e1.x, e2.x, e3.x);
            *reinterpret_cast<float4*>(o + nn + (size_t)iy * n + ix) = make_float4(e0.y, e1.y, e2.y, e3.y);
        }
    } else if (r < n && c < n) {
        *reinterpret_cast<float4*>(o + (size_t)r * n + c) =
            make_float4(a[0][0].val(), a[0][1].val(), a[0][2].val(), a[0][3].val());
        *reinterpret_cast<float4*>(o + nn + (size_t)r * n + c) =
            make_float4(a[1][0].val(), a[1][1].val(), a[1][2].val(), a[1][3].val());
    }
}

// Stage 2: out = sum over groups (+ alpha grad^T W grad v + nu v when v given);
// per-block partial of <dotv, out> when dotv given.
template <typename T, typename TP, bool KAHAN>
__global__ void reduce_groups_kernel(RedArgs<T> a, const TP* __restrict__ in2) {
    if (a.skip && *a.skip) return;
    const size_t nn = (size_t)a.n * a.n;
    double acc = 0.0;
    const double nu = a.nu_dev ? *a.nu_dev : a.nu;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * nn; e += (size_t)gridDim.x * blockDim.x) {
        const int f = e >= nn;
        const size_t i = e - f * nn;
        Acc<T, KAHAN> s;
        s.init();
        for (int g = 0; g < a.groups; ++g) s.add((T)in2[(size_t)g * 2 * nn + e]);
        T val = s.val();
        if (a.v) {
            const int iy = (int)(i / a.n), ix = (int)(i - (size_t)iy * a.n);
            const T* vf = a.v + f * nn;
            val += reg_at(vf, f ? a.Wm : a.Wl, (T)(f ? a.alpha_m : a.alpha_l), a.n, ix, iy);
            if (a.gmask) {  // geometry prior of Eq. (6): 2 alpha (1 - M)^2 (v - c)
                const T om = T(1) - a.gmask[i];
                const T c = (a.geo_offset && f) ? (T)a.geo_cm : T(0);
                val += (T)(2.0 * (f ? a.geo_m : a.geo_l)) * om * om * (vf[i] - c);
            }
            val += (T)nu * vf[i];
        }
        a.out[e] = val;
        if (a.dotv) acc += (double)a.dotv[e] * (double)val;
    }
    if (a.dotv) {
        double s = block_sum(acc);
        if (threadIdx.x == 0) a.part[blockIdx.x] = s;
    }
}

template <typename T, typename TP>
void reduce_views(const TP* gpart, int n, int n_views, int n0, int groups, TP* part2, const RedArgs<T>& ra,
                  bool kahan, cudaStream_t st) {
    const int tiles_x = (n + 31) / 32;
    // groups per orientation in proportion to its views, at least one for each present
    int g0 = n0 <= 0 ? 0 : (n0 >= n_views ? groups : (int)((long long)groups * n0 / n_views));
    if (n0 > 0 && n0 < n_views) g0 = std::min(std::max(g0, 1), groups - 1);
    dim3 block(32, 8);
    const int grid = tiles_x * tiles_x * groups;
    bool vec4 = false;
    if constexpr (std::is_same<TP, float>::value) {
        vec4 = n % 4 == 0;  // then partial images and their rows start on 16-byte boundaries
        if (vec4 && kahan)
            reduce_views4_kernel<true><<<grid, block, 0, st>>>(gpart, n, n_views, n0, groups, g0, part2, ra.skip);
        else if (vec4)
            reduce_views4_kernel<false><<<grid, block, 0, st>>>(gpart, n, n_views, n0, groups, g0, part2, ra.skip);
    }
    if (!vec4 && kahan)
        reduce_views_kernel<TP, true><<<grid, block, 0, st>>>(gpart, n, n_views, n0, groups, g0, part2, ra.skip);
    else if (!vec4)
        reduce_views_kernel<TP, false><<<grid, block, 0, st>>>(gpart, n, n_views, n0, groups, g0, part2, ra.skip);
    RedArgs<T> r2 = ra;
    r2.groups = groups;
    if (kahan)
        reduce_groups_kernel<T, TP, true><<<kRedBlocks, 256, 0, st>>>(r2, part2);
    else
        reduce_groups_kernel<T, TP, false><<<kRedBlocks, 256, 0, st>>>(r2, part2);
    note_launch(2);
}
template void reduce_views<float, float>(const float*, int, int, int, int, float*, const RedArgs<float>&, bool,
                                         cudaStream_t);
template void reduce_views<double, double>(const double*, int, int, int, int, double*, const RedArgs<double>&, bool,
                                           cudaStream_t);
template void reduce_views<double, float>(const float*, int, int, int, int, float*, const RedArgs<double>&, bool,
                                          cudaStream_t);

// ------------------------------------------------------------------ elementwise
template <typename T>
__global__ void sub_dot_kernel(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, size_t m,
                               double* __restrict__ part, const int* skip) {
    if (skip && *skip) return;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        T d = a[i] - b[i];
        out[i] = d;
        acc += (double)d * (double)d;
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = s;
}
template <typename T>
void sub_dot(const T* a, const T* b, T* out, size_t m, double* part, const int* skip, cudaStream_t st) {
    sub_dot_kernel<T><<<kRedBlocks, 256, 0, st>>>(a, b, out, m, part, skip);
    note_launch();
}
template void sub_dot<float>(const float*, const float*, float*, size_t, double*, const int*, cudaStream_t);
template void sub_dot<double>(const double*, const double*, double*, size_t, double*, const int*, cudaStream_t);

// Component c (0: lambda, 1: mu) of the Euclidean projection of the pixel pair (zl, zm)
// onto the constraint set f.  The box clamp is the answer when it meets the linear bound
// (or there is none); otherwise the bound is active and the answer is the nearest point
// of its segment inside the box, lambda = k t + b, mu = t, with t the foot of the
// perpendicular ((zl - b) k + zm) / (k^2 + 1) clamped to [0, t_hi].
template <typename T>
__device__ __forceinline__ T project_comp(T zl, T zm, int c, const Feas& f) {
    const T lh = (T)f.lmax, mh = (T)f.mmax;
    T pl = zl < T(0) ? T(0) : (zl > lh ? lh : zl);
    T pm = zm < T(0) ? T(0) : (zm > mh ? mh : zm);
    const T k = (T)f.k, b = (T)f.b;
    if (f.lin && pl - k * pm > b) {
        T t = ((zl - b) * k + zm) / (T)f.den;
        t = t < T(0) ? T(0) : (t > (T)f.t_hi ? (T)f.t_hi : t);
        pl = k * t + b;
        pm = t;
    }
    return c ? pm : pl;
}

// (lambda, mu) = P(lambda, mu) in place, one thread per pixel
template <typename T>
__global__ void project_kernel(T* __restrict__ ul, T* __restrict__ um, size_t nn, Feas f) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        const T zl = ul[i], zm = um[i];
        ul[i] = project_comp(zl, zm, 0, f);
        um[i] = project_comp(zl, zm, 1, f);
    }
}
template <typename T>
void project_pair(T* lam, T* mu, size_t nn, const Feas& f, cudaStream_t st) {
    project_kernel<T><<<kRedBlocks, 256, 0, st>>>(lam, mu, nn, f);
    note_launch();
}
template <typename T>
void project_set(T* u, size_t nn, const Feas& f, cudaStream_t st) {
    project_pair<T>(u, u + nn, nn, f, st);
}
template void project_set<float>(float*, size_t, const Feas&, cudaStream_t);
template void project_pair<float>(float*, float*, size_t, const Feas&, cudaStream_t);
template void project_set<double>(double*, size_t, const Feas&, cudaStream_t);
template void project_pair<double>(double*, double*, size_t, const Feas&, cudaStream_t);

template <typename T>
__global__ void fill_kernel(T* __restrict__ u, size_t m, double v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        u[i] = (T)v;
}
template <typename T>
void fill(T* u, size_t m, double v, cudaStream_t st) {
    fill_kernel<T><<<kRedBlocks, 256, 0, st>>>(u, m, v);
    note_launch();
}
template void fill<float>(float*, size_t, double, cudaStream_t);
template void fill<double>(double*, size_t, double, cudaStream_t);

// ---------------------------------------------------------------------- CG
// x = 0, res = b, p = b; partial <b, b>
template <typename T>
__global__ void cg_init_kernel(const T* __restrict__ b, T* __restrict__ x, T* __restrict__ res,
                               T* __restrict__ p, size_t m, double scale_b, double tol,
                               double* __restrict__ part, CgState* cg) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        T v = (T)scale_b * b[i];
        x[i] = T(0);
        res[i] = v;
        p[i] = v;
        acc += (double)v * (double)v;
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cg->stop = 0;
        cg->iters = 0;
        cg->tol = tol;
    }
}

__global__ void cg_finish_init_kernel(const double* __restrict__ part, CgState* cg) {
    const double s = warp_sum_partials(part);
    if (threadIdx.x) return;
    cg->rr = s;
    cg->bnorm = sqrt(s);
    cg->stop = !(cg->bnorm > 0.0) || !isfinite(s);
    cg->iters = 0;
}

// The solve's stop flag as one value per block.  Block 0 of the fused CG kernels below
// may set the flag while other blocks of the same launch are starting: each block reads
// it once, so that all its threads take the same branch around the block barriers.
__device__ __forceinline__ bool block_stopped(const CgState* cg) {
    __shared__ int s;
    if (threadIdx.x == 0 && threadIdx.y == 0) s = cg->stop;
    __syncthreads();
    return s != 0;
}

// The kRedBlocks partials summed by warp 0 of the block in the fixed order of
// warp_sum_partials (every block obtains the same value) and shared with the block.
__device__ __forceinline__ double block_partials(const double* __restrict__ part) {
    __shared__ double v;
    if (threadIdx.y == 0 && threadIdx.x < 32) {
        const double s = warp_sum_partials(part);
        if (threadIdx.x == 0) v = s;
    }
    __syncthreads();
    return v;
}

// CG step fused with the finish of <p, q>: every block forms alpha = rr / <p, q> from the
// partials part_pq itself; x += alpha p, res -= alpha q, per-block partials of |res|^2 into
// part_rr (a separate buffer: other blocks may still be reading part_pq).  Block 0 records
// pq, alpha and rr_prev = rr for the p update; <p, q> <= 0 or non-finite stops the solve.
template <typename T>
__global__ void cg_step_kernel(T* __restrict__ x, T* __restrict__ res, const T* __restrict__ p,
                               const T* __restrict__ q, size_t m, const double* __restrict__ part_pq,
                               double* __restrict__ part_rr, CgState* cg) {
    if (block_stopped(cg)) return;
    const double pq = block_partials(part_pq);
    const double rr = cg->rr;
    const bool bad = !(pq > 0.0) || !isfinite(pq);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cg->pq = pq;
        if (bad) cg->stop = 1;
        else {
            cg->alpha = rr / pq;
            cg->rr_prev = rr;
        }
    }
    if (bad) return;
    const T al = (T)(rr / pq);
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        x[i] += al * p[i];
        T r = res[i] - al * q[i];
        res[i] = r;
        acc += (double)r * (double)r;
    }
    double sum = block_sum(acc);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = sum;
}

// Direction update fused with the finish of |res|^2 and the packing of p for the next
// JVP: every block forms s = |res|^2 from the partials; the iteration counts, and stops
// (p untouched) when sqrt(s) <= tol |b| or s is not finite; otherwise
// p = res + (s / rr_prev) p on the block's 32 x 32 tile of both fields, written planar and
// in the two padded layouts of pack_kernel.  Block 0 records iters, rr and beta.
template <typename T, typename TW>
__global__ void cg_dir_pack_kernel(T* __restrict__ p, const T* __restrict__ res, const double* __restrict__ part_rr,
                                   CgState* cg, int n, int P, T mu_scale, typename Vec2<TW>::type* __restrict__ out_n,
                                   typename Vec2<TW>::type* __restrict__ out_t) {
    using T2 = typename Vec2<TW>::type;
    if (block_stopped(cg)) return;
    const double s = block_partials(part_rr);
    const double rp = cg->rr_prev;
    const bool done = sqrt(s) <= cg->tol * cg->bnorm || !isfinite(s);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        cg->iters += 1;
        cg->rr = s;
        if (!done) cg->beta = s / rp;
    }
    if (done) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) cg->stop = 1;
        return;
    }
    const T be = (T)(s / rp);
    const size_t nn = (size_t)n * n;
    __shared__ T2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int iy = by + k, ix = bx + threadIdx.x;
        if (iy < n && ix < n) {
            const size_t i = (size_t)iy * n + ix;
            const T pl = res[i] + be * p[i];
            const T pm = res[nn + i] + be * p[nn + i];
            p[i] = pl;
            p[nn + i] = pm;
            const T2 v = mk2((TW)pl, (TW)(mu_scale * pm));
            out_n[(size_t)(iy + 1) * P + ix + 1] = v;
            tile[k][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int ix = bx + k, iy = by + threadIdx.x;
        if (iy < n && ix < n) out_t[(size_t)(ix + 1) * P + iy + 1] = tile[threadIdx.x][k];
    }
}

template <typename T>
void cg_step(T* x, T* res, const T* p, const T* q, size_t m, const double* part_pq, double* part_rr, CgState* cg,
             cudaStream_t st) {
    cg_step_kernel<T><<<kRedBlocks, 256, 0, st>>>(x, res, p, q, m, part_pq, part_rr, cg);
    note_launch();
}
template <typename T, typename TW>
void cg_dir_pack(T* p, const T* res, const double* part_rr, CgState* cg, int n, int P, double mu_scale, void* out_n,
                 void* out_t, cudaStream_t st) {
    dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
    cg_dir_pack_kernel<T, TW><<<grid, block, 0, st>>>(p, res, part_rr, cg, n, P, (T)mu_scale,
                                                      (typename Vec2<TW>::type*)out_n, (typename Vec2<TW>::type*)out_t);
    note_launch();
}
template void cg_step<float>(float*, float*, const float*, const float*, size_t, const double*, double*, CgState*,
                             cudaStream_t);
template void cg_step<double>(double*, double*, const double*, const double*, size_t, const double*, double*,
                              CgState*, cudaStream_t);
template void cg_dir_pack<float, float>(float*, const float*, const double*, CgState*, int, int, double, void*,
                                        void*, cudaStream_t);
template void cg_dir_pack<double, double>(double*, const double*, const double*, CgState*, int, int, double, void*,
                                          void*, cudaStream_t);
template void cg_dir_pack<double, float>(double*, const double*, const double*, CgState*, int, int, double, void*,
                                         void*, cudaStream_t);

template <typename T>
void cg_init(const T* b, T* x, T* res, T* p, size_t m, double scale_b, double tol, double* part, CgState* cg,
             cudaStream_t st) {
    cg_init_kernel<T><<<kRedBlocks, 256, 0, st>>>(b, x, res, p, m, scale_b, tol, part, cg);
    note_launch();
    cg_finish_init_kernel<<<1, 32, 0, st>>>(part, cg);
    note_launch();
}
template void cg_init<float>(const float*, float*, float*, float*, size_t, double, double, double*, CgState*, cudaStream_t);
template void cg_init<double>(const double*, double*, double*, double*, size_t, double, double, double*, CgState*, cudaStream_t);

// ------------------------------------------------------------- trust region
// ut = P(u + x), s = ut - u (P: projection onto the constraint set)
template <typename T>
__global__ void lm_step_kernel(const T* __restrict__ u, const T* __restrict__ x, T* __restrict__ ut,
                               T* __restrict__ s, size_t nn, Feas f) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 2 * nn; i += (size_t)gridDim.x * blockDim.x) {
        T v = u[i] + x[i];
        if (f.lin) {  // the pair of this pixel: the other component is at i -/+ nn
            const size_t o = i < nn ? i + nn : i - nn;
            const T w = u[o] + x[o];
            v = i < nn ? project_comp(v, w, 0, f) : project_comp(w, v, 1, f);
        } else {
            const T hi = (T)(i < nn ? f.lmax : f.mmax);
            v = v < T(0) ? T(0) : (v > hi ? hi : v);
        }
        ut[i] = v;
        s[i] = v - u[i];
    }
}
template <typename T>
void lm_step(const T* u, const T* x, T* ut, T* s, size_t nn, const Feas& f, cudaStream_t st) {
    lm_step_kernel<T><<<kRedBlocks, 256, 0, st>>>(u, x, ut, s, nn, f);
    note_launch();
}
template void lm_step<float>(const float*, const float*, float*, float*, size_t, const Feas&, cudaStream_t);
template void lm_step<double>(const double*, const double*, double*, double*, size_t, const Feas&, cudaStream_t);

// partials of <s, g> (part_a) and <s, H s> (part_b), H = alpha grad^T W grad per field
template <typename T>
__global__ void lm_model_kernel(const T* __restrict__ s, const T* __restrict__ g, const T* __restrict__ Wl,
                                const T* __restrict__ Wm, int n, double al, double am,
                                double* __restrict__ part_a, double* __restrict__ part_b,
                                const T* __restrict__ gmask, double geo_l, double geo_m) {
    const size_t nn = (size_t)n * n;
    double a = 0.0, b = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * nn; e += (size_t)gridDim.x * blockDim.x) {
        const int f = e >= nn;
        const size_t i = e - f * nn;
        const int iy = (int)(i / n), ix = (int)(i - (size_t)iy * n);
        const T* sf = s + f * nn;
        T hs = reg_at(sf, f ? Wm : Wl, (T)(f ? am : al), n, ix, iy);
        a += (double)s[e] * (double)g[e];
        b += (double)sf[i] * (double)hs;
        if (gmask) {  // s^T (2 alpha (1 - M)^2) s of the geometry prior
            const double om = 1.0 - (double)gmask[i];
            b += 2.0 * (f ? geo_m : geo_l) * om * om * (double)sf[i] * (double)sf[i];
        }
    }
    double sa = block_sum(a);
    double sb = block_sum(b);
    if (threadIdx.x == 0) {
        part_a[blockIdx.x] = sa;
        part_b[blockIdx.x] = sb;
    }
}
template <typename T>
void lm_model(const T* s, const T* g, const T* Wl, const T* Wm, int n, double al, double am, double* pa,
              double* pb, cudaStream_t st, const T* gmask, double geo_l, double geo_m) {
    lm_model_kernel<T><<<kRedBlocks, 256, 0, st>>>(s, g, Wl, Wm, n, al, am, pa, pb, gmask, geo_l, geo_m);
    note_launch();
}
template void lm_model<float>(const float*, const float*, const float*, const float*, int, double, double, double*,
                              double*, cudaStream_t, const float*, double, double);
template void lm_model<double>(const double*, const double*, const double*, const double*, int, double, double,
                               double*, double*, cudaStream_t, const double*, double, double);

// One thread: predicted and actual decrease, rho (Eq. (12)), acceptance, nu update.
__global__ void lm_decide_kernel(LmState* L, LmParamsDev P) {
    if (threadIdx.x || blockIdx.x) return;
    double pred = -L->sg - 0.5 * L->JsJs - 0.5 * L->sHs;
    double ft = 0.5 * L->rtrt + L->Rl + L->Rm;
    double ared = L->f - ft;
    double rho = (pred > 0.0 && isfinite(ft)) ? ared / pred : -INFINITY;
    int acc = rho > P.eta;
    if (acc) L->f = ft;
    double nu = L->nu;
    if (rho < P.rho_lo) nu *= P.nu_up;
    else if (rho > P.rho_hi) nu *= P.nu_down;
    nu = fmin(fmax(nu, P.nu_min * L->nu0), P.nu_max * L->nu0);
    L->nu = nu;
    L->accept = acc;
    L->no_grad = !acc;
    int k = L->iter;
    if (k < PGET_TRACE) {
        L->tr_f[k] = L->f;
        L->tr_rho[k] = rho;
        L->tr_nu[k] = nu;
        L->tr_pred[k] = pred;
        L->tr_ared[k] = ared;
        L->tr_acc[k] = acc;
        L->tr_cg[k] = L->cg.iters;
    }
    L->accepted += acc;
    L->cg_total += L->cg.iters;
    L->iter = k + 1;
}
void lm_decide(LmState* L, const LmParamsDev& P, cudaStream_t st) { lm_decide_kernel<<<1, 32, 0, st>>>(L, P); }

// f = 1/2 |r|^2 + R_l + R_m from the finished sums (initial objective)
__global__ void lm_init_f_kernel(LmState* L, double nu0_scale) {
    if (threadIdx.x || blockIdx.x) return;
    L->f = 0.5 * L->rtrt + L->Rl + L->Rm;
    L->f0 = L->f;
    double nu0 = (L->gg > 0.0) ? nu0_scale * L->JsJs / L->gg : 1.0;
    if (!(nu0 > 0.0) || !isfinite(nu0)) nu0 = 1.0;
    L->nu0 = nu0;
    L->nu = nu0;
    L->iter = 0;
    L->accepted = 0;
    L->cg_total = 0;
    L->accept = 0;
    L->no_grad = 1;
}
void lm_init_f(LmState* L, double nu0_scale, cudaStream_t st) { lm_init_f_kernel<<<1, 32, 0, st>>>(L, nu0_scale); }

// f at the current iterate from its data term and prior values (after new prior weights)
__global__ void lm_refresh_f_kernel(LmState* L) {
    if (threadIdx.x || blockIdx.x) return;
    L->f = 0.5 * L->rtrt + L->Rl + L->Rm;
}
void lm_refresh_f(LmState* L, cudaStream_t st) {
    lm_refresh_f_kernel<<<1, 32, 0, st>>>(L);
    note_launch();
}

// ------------------------------------------------------- gradient projection
// min_s <g, s> + 1/2 s^T A s subject to u + s in the constraint set (A = J^T J + H + nu I),
// from s = 0: d = P(u + s - alpha grad q) - u - s with P the projection onto the set (box,
// and the linear bound if set), exact line search on [0, 1] for the quadratic,
// alternating Barzilai-Borwein lengths; stop on the unit-step projected gradient.
template <typename T>
__global__ void sgp_init_kernel(const T* __restrict__ g, T* __restrict__ gq, T* __restrict__ x, size_t m, double tol,
                                CgState* cg) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        x[i] = T(0);
        gq[i] = g[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cg->stop = 0;
        cg->iters = 0;
        cg->tol = tol;
        cg->alpha = 1.0;
        cg->bnorm = -1.0;
    }
}

template <typename T>
__global__ void sgp_dir_kernel(const T* __restrict__ u, const T* __restrict__ x, const T* __restrict__ gq,
                               T* __restrict__ d, size_t nn, Feas f, double* __restrict__ p_pg,
                               double* __restrict__ p_gd, double* __restrict__ p_dd, const CgState* cg) {
    if (cg->stop) return;
    const T al = (T)cg->alpha;
    double a = 0.0, b = 0.0, c = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 2 * nn; i += (size_t)gridDim.x * blockDim.x) {
        const T ui = u[i], xi = x[i], gi = gq[i];
        T v1 = ui + xi - gi;
        T v = ui + xi - al * gi;
        if (f.lin) {  // project the pixel's pair; the other component is at i -/+ nn
            const size_t o = i < nn ? i + nn : i - nn;
            const T uo = u[o], xo = x[o], go = gq[o];
            const T w1 = uo + xo - go, w = uo + xo - al * go;
            v1 = i < nn ? project_comp(v1, w1, 0, f) : project_comp(w1, v1, 1, f);
            v = i < nn ? project_comp(v, w, 0, f) : project_comp(w, v, 1, f);
        } else {
            const T hi = (T)(i < nn ? f.lmax : f.mmax);
            v1 = v1 < T(0) ? T(0) : (v1 > hi ? hi : v1);
            v = v < T(0) ? T(0) : (v > hi ? hi : v);
        }
        const T z1 = (v1 - ui) - xi;
        const T di = (v - ui) - xi;
        d[i] = di;
        a += (double)z1 * (double)z1;
        b += (double)gi * (double)di;
        c += (double)di * (double)di;
    }
    const double sa = block_sum(a);
    const double sb = block_sum(b);
    const double sc = block_sum(c);
    if (threadIdx.x == 0) {
        p_pg[blockIdx.x] = sa;
        p_gd[blockIdx.x] = sb;
        p_dd[blockIdx.x] = sc;
    }
}

__global__ void sgp_check_kernel(const double* __restrict__ p_pg, const double* __restrict__ p_gd,
                                 const double* __restrict__ p_dd, CgState* cg) {
    if (cg->stop) return;
    const double pg2 = warp_sum_partials(p_pg);
    const double gd = warp_sum_partials(p_gd);
    const double dd = warp_sum_partials(p_dd);
    if (threadIdx.x) return;
    const double pg = sqrt(pg2);
    if (cg->bnorm < 0.0) cg->bnorm = pg;
    cg->rr = pg;
    cg->pq = gd;
    cg->dd = dd;
    if (pg <= cg->tol * cg->bnorm || cg->bnorm == 0.0 || !(gd < 0.0)) cg->stop = 1;
}

__global__ void sgp_step_kernel(const double* __restrict__ p_dAd, const double* __restrict__ p_AdAd, CgState* cg) {
    if (cg->stop) return;
    const double dAd = warp_sum_partials(p_dAd);
    const double AdAd = warp_sum_partials(p_AdAd);
    if (threadIdx.x) return;
    if (!(dAd > 0.0)) {
        cg->stop = 1;
        return;
    }
    double ls = -cg->pq / dAd;
    if (ls > 1.0) ls = 1.0;
    cg->beta = ls;
    cg->iters += 1;
    const double an = (cg->iters % 2) ? cg->dd / dAd : dAd / AdAd;
    cg->alpha = fmin(fmax(an, 1e-10), 1e10);
}

template <typename T>
__global__ void sgp_update_kernel(T* __restrict__ x, T* __restrict__ gq, const T* __restrict__ d,
                                  const T* __restrict__ Ad, size_t m, const CgState* cg) {
    if (cg->stop) return;
    const T ls = (T)cg->beta;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        x[i] += ls * d[i];
        gq[i] += ls * Ad[i];
    }
}

template <typename T>
void sgp_init(const T* g, T* gq, T* x, size_t m, double tol, CgState* cg, cudaStream_t st) {
    sgp_init_kernel<T><<<kRedBlocks, 256, 0, st>>>(g, gq, x, m, tol, cg);
    note_launch();
}
template <typename T>
void sgp_dir(const T* u, const T* x, const T* gq, T* d, size_t nn, const Feas& f, double* p_pg,
             double* p_gd, double* p_dd, CgState* cg, cudaStream_t st) {
    sgp_dir_kernel<T><<<kRedBlocks, 256, 0, st>>>(u, x, gq, d, nn, f, p_pg, p_gd, p_dd, cg);
    sgp_check_kernel<<<1, 32, 0, st>>>(p_pg, p_gd, p_dd, cg);
    note_launch(2);
}
void sgp_step(const double* p_dAd, const double* p_AdAd, CgState* cg, cudaStream_t st) {
    sgp_step_kernel<<<1, 32, 0, st>>>(p_dAd, p_AdAd, cg);
    note_launch();
}
template <typename T>
void sgp_update(T* x, T* gq, const T* d, const T* Ad, size_t m, const CgState* cg, cudaStream_t st) {
    sgp_update_kernel<T><<<kRedBlocks, 256, 0, st>>>(x, gq, d, Ad, m, cg);
    note_launch();
}
template void sgp_init<float>(const float*, float*, float*, size_t, double, CgState*, cudaStream_t);
template void sgp_init<double>(const double*, double*, double*, size_t, double, CgState*, cudaStream_t);
template void sgp_dir<float>(const float*, const float*, const float*, float*, size_t, const Feas&, double*, double*,
                             double*, CgState*, cudaStream_t);
template void sgp_dir<double>(const double*, const double*, const double*, double*, size_t, const Feas&, double*,
                              double*, double*, CgState*, cudaStream_t);
template void sgp_update<float>(float*, float*, const float*, const float*, size_t, const CgState*, cudaStream_t);
template void sgp_update<double>(double*, double*, const double*, const double*, size_t, const CgState*, cudaStream_t);

// conditional copy (accepted trial becomes the iterate)
template <typename T>
__global__ void copy_if_kernel(T* __restrict__ dst, const T* __restrict__ src, size_t m, const int* flag) {
    if (!*flag) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
template <typename T>
void copy_if(T* dst, const T* src, size_t m, const int* flag, cudaStream_t st) {
    copy_if_kernel<T><<<kRedBlocks, 256, 0, st>>>(dst, src, m, flag);
    note_launch();
}
template void copy_if<float>(float*, const float*, size_t, const int*, cudaStream_t);
template void copy_if<double>(double*, const double*, size_t, const int*, cudaStream_t);
template void copy_if<float2>(float2*, const float2*, size_t, const int*, cudaStream_t);
template void copy_if<double2>(double2*, const double2*, size_t, const int*, cudaStream_t);

// scale: y = c y (in place)
template <typename T>
__global__ void scale_kernel(T* __restrict__ y, size_t m, double c) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (T)c * y[i];
}
template <typename T>
void scale(T* y, size_t m, double c, cudaStream_t st) {
    scale_kernel<T><<<kRedBlocks, 256, 0, st>>>(y, m, c);
    note_launch();
}
template void scale<float>(float*, size_t, double, cudaStream_t);
template void scale<double>(double*, size_t, double, cudaStream_t);

template <typename T>
__global__ void fill_ratio_kernel(T* __restrict__ u, size_t m, const double* num, const double* den, double hi) {
    const double d = *den;
    double c = d > 0.0 ? *num / d : 0.0;
    c = c < 0.0 ? 0.0 : (c > hi ? hi : c);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        u[i] = (T)c;
}
template <typename T>
void fill_ratio(T* u, size_t m, const double* num, const double* den, double hi, cudaStream_t st) {
    fill_ratio_kernel<T><<<kRedBlocks, 256, 0, st>>>(u, m, num, den, hi);
    note_launch();
}
template void fill_ratio<float>(float*, size_t, const double*, const double*, double, cudaStream_t);
template void fill_ratio<double>(double*, size_t, const double*, const double*, double, cudaStream_t);

}  // namespace pget
