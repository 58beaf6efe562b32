// walk.cu -- the ray kernels of the hot path: forward model, JVP and the scatter-free VJP.
//
// One CTA per view (angle, bank); one thread per ray slot.  The canonical image of the
// view (normal or transposed layout, rows possibly reversed so rays climb in Y) is
// streamed through shared memory in chunks of Yc base rows, starting at the detector
// side; each thread walks its ray from the detector end toward the far end, so the
// attenuation sum E_j = h (mu_j/2 + sum_{i>j} mu_i) of Eq. (1) is a running suffix sum.
//
//   forward (Eq. (1), sampled as Eq. (5)):  q = h sum_j lambda_j exp(-E_j)
//   JVP (Eq. (2)):                          q' = h sum_j exp(-E_j) (dl_j - lambda_j dE_j)
//   VJP (adjoint of Eq. (2)):  per sample   g_lambda = rho h exp(-E_j)
//                                           g_mu = -rho h^2 (sum_{l<j} lambda_l e_l + lambda_j e_j / 2)
//     with rho = sum of w_k r over the sub-rays on this slot; the far-side prefix is the
//     ray total (from the forward pass) minus the detector-side suffix.  The samples of a
//     chunk are kept in shared memory and every pixel of the chunk's rows then GATHERS
//     the bilinear contributions of the samples whose footprint covers it (no atomics).
//     Pixel rows shared by two chunks are carried in shared memory.  Each view writes
//     its own partial image; reduce_views sums them in a fixed order.
#include <atomic>
#include <cstdio>

#include "kernels.cuh"

namespace pget {

static std::atomic<long long> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ray clipping: conservative j range of samples whose base pixel can be inside
// [-1, n-1]^2; the exact per-sample test inside the walk decides
__device__ __forceinline__ void clip_ray(const ViewDev& v, int i, int n, int T, int* jlo, int* jhi) {
    double X0 = v.X00d + i * v.dXrd, Y0 = v.Y00d + i * v.dYrd;
    double lo = 0.0, hi = T - 1.0;
    lo = fmax(lo, ceil((-1.0 - Y0) / v.dYsd) - 1.0);
    hi = fmin(hi, floor((n - Y0) / v.dYsd) + 1.0);
    if (fabs(v.dXsd) > 1e-9) {
        double a = (-1.0 - X0) / v.dXsd, b = (n - X0) / v.dXsd;
        if (a > b) {
            double t = a;
            a = b;
            b = t;
        }
        lo = fmax(lo, ceil(a) - 1.0);
        hi = fmin(hi, floor(b) + 1.0);
    } else if (X0 < -1.0 - 1e-6 || X0 > n + 1e-6) {
        hi = lo - 1.0;
    }
    if (hi < lo) {
        *jlo = 0;
        *jhi = -1;
    } else {
        *jlo = (int)lo;
        *jhi = (int)hi;
    }
}

// copy canonical rows [row_lo, row_lo + nrows) of a padded layout into shared memory
template <typename T2>
__device__ __forceinline__ void stage_rows(T2* __restrict__ dst, const T2* __restrict__ src, int P,
                                           int n, int flipped, int row_lo, int nrows) {
    const int total = nrows * P;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int rr = e / P, col = e - rr * P;
        int r = row_lo + rr;
        int gr = (flipped ? (n - 1 - r) : r) + 1;
        dst[e] = src[(size_t)gr * P + col];
    }
}

template <typename T, bool KAHAN, int MODE>
__global__ void __launch_bounds__(kMaxSlots) walk_kernel(WalkArgs A) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char sm[];
    if (A.stop && *A.stop) return;
    const int v = blockIdx.x;
    const ViewDev vp = A.views[v];
    const int n = A.n, P = A.P, Yc = A.Yc, ns = vp.n_slots, tid = threadIdx.x;
    const int nth = blockDim.x;
    const bool active = tid < ns;
    const T h = (T)A.h;

    size_t off = 0;
    T2* cu = (T2*)(sm + off);
    off += sizeof(T2) * (size_t)(Yc + 1) * P;
    T2* cp = nullptr;
    if constexpr (MODE == kJvp) {
        cp = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)(Yc + 1) * P;
    }
    T* sval = (T*)(sm + off);
    off += sizeof(T2) * (size_t)nth;  // T2-sized slots keep the next arrays aligned
    T2 *SBg = nullptr, *SBa = nullptr, *carry0 = nullptr, *carry1 = nullptr;
    int *SBi = nullptr, *scnt = nullptr;
    float* sYf = nullptr;
    const int cap = A.sb_cap;
    if constexpr (MODE == kVjp) {
        SBg = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)cap * nth;
        SBa = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)cap * nth;
        carry0 = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)n;
        carry1 = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)n;
        SBi = (int*)(sm + off);
        off += sizeof(int) * (size_t)cap * nth;
        scnt = (int*)(sm + off);
        off += sizeof(int) * (size_t)nth;
        sYf = (float*)(sm + off);
        off += sizeof(float) * (size_t)nth;
    }

    const T2* ug = (const T2*)A.u_img[vp.transposed];
    const T2* pg = (MODE == kJvp) ? (const T2*)A.p_img[vp.transposed] : nullptr;

    int jlo = 0, jhi = -1;
    if (active) clip_ray(vp, tid, n, A.T, &jlo, &jhi);
    int j = jhi;
    Pos<T> pos;
    pos.init(vp, active ? tid : 0, j);
    Acc<T, KAHAN> S, q, dS;
    S.init();
    q.init();
    dS.init();
    T rho = T(0), Utot = T(0);
    if constexpr (MODE == kVjp) {
        if (active) {
            const int q0 = A.src_off[vp.bank * A.max_slots + tid];
            const int q1 = A.src_off[vp.bank * A.max_slots + tid + 1];
            const T* r = (const T*)A.r_in + (size_t)vp.angle * A.n_det;
            T acc = T(0);
            for (int e = q0; e < q1; ++e) acc += (T)A.src_w[e] * r[A.src_det[e]];
            rho = acc;
            Utot = ((const T*)A.slot_val)[(size_t)v * A.max_slots + tid];
        }
    }
    // gather geometry of this view (float is enough to bound candidates)
    const float X00f = (float)vp.X00d, Y00f = (float)vp.Y00d;
    const float dXrf = (float)vp.dXrd, dYrf = (float)vp.dYrd;
    const float invR2 = 1.0f / (dXrf * dXrf + dYrf * dYrf);
    const float wI = (fabsf(dXrf) + fabsf(dYrf)) * invR2 + 0.01f;
    const float invdY = (float)(1.0 / vp.dYsd);

    for (int ck = 0; ck < A.nchunks; ++ck) {
        const int row_hi = n - 1 - ck * Yc;
        const int row_lo = max(-1, row_hi - Yc + 1);
        const int nrows = row_hi - row_lo + 2;
        __syncthreads();
        stage_rows(cu, ug, P, n, vp.flipped, row_lo, nrows);
        if constexpr (MODE == kJvp) stage_rows(cp, pg, P, n, vp.flipped, row_lo, nrows);
        __syncthreads();
        int cnt = 0;
        if (active) {
            while (j >= jlo) {
                const int iy0 = pos.iy();
                if (iy0 < row_lo) break;
                const int ix0 = pos.ix();
                if (iy0 <= row_hi && ix0 >= -1 && ix0 <= n - 1) {
                    const T ax = pos.ax(), ay = pos.ay();
                    const int o = (iy0 - row_lo) * P + ix0 + 1;
                    const T2 a00 = cu[o], a10 = cu[o + 1], a01 = cu[o + P], a11 = cu[o + P + 1];
                    const T w11 = ax * ay, w10 = ax - w11, w01 = ay - w11;
                    const T w00 = (T(1) - ax) - w01;
                    const T l = w00 * a00.x + w10 * a10.x + w01 * a01.x + w11 * a11.x;
                    const T m = w00 * a00.y + w10 * a10.y + w01 * a01.y + w11 * a11.y;
                    const T E = h * (S.val() + T(0.5) * m);
                    const T at = exp_(-E);
                    if constexpr (MODE == kFwd) {
                        q.add(l * at);
                    } else if constexpr (MODE == kJvp) {
                        const T2 b00 = cp[o], b10 = cp[o + 1], b01 = cp[o + P], b11 = cp[o + P + 1];
                        const T dl = w00 * b00.x + w10 * b10.x + w01 * b01.x + w11 * b11.x;
                        const T dm = w00 * b00.y + w10 * b10.y + w01 * b01.y + w11 * b11.y;
                        const T dE = h * (dS.val() + T(0.5) * dm);
                        q.add(at * (dl - l * dE));
                        dS.add(dm);
                    } else {
                        const T la = l * at;
                        const T Qh = (Utot - q.val()) - T(0.5) * la;
                        const T gl = rho * h * at;
                        const T gm = -rho * h * h * Qh;
                        if (cnt == 0) sYf[tid] = pos.yf();
                        if (cnt < cap) {
                            SBg[cnt * nth + tid] = mk2(gl, gm);
                            SBa[cnt * nth + tid] = mk2(ax, ay);
                            SBi[cnt * nth + tid] = (ix0 + 1) | ((iy0 + 1) << 16);
                        } else {
                            atomicOr(A.err, 1);
                        }
                        ++cnt;
                        q.add(la);
                    }
                    S.add(m);
                }
                --j;
                pos.back();
            }
        }
        if constexpr (MODE == kVjp) {
            scnt[tid] = active ? min(cnt, cap) : 0;
            __syncthreads();
            const int r0 = max(row_lo, 0), r1 = min(row_hi + 1, n - 1);
            const int nout = (r1 - r0 + 1) * n;
            T2* carry_rd = (ck & 1) ? carry0 : carry1;
            T2* carry_wr = (ck & 1) ? carry1 : carry0;
            T* gp = (T*)A.gpart + (size_t)v * 2 * n * n;
            for (int e = tid; e < nout; e += nth) {
                const int Yr = r0 + e / n, Xc = e - (e / n) * n;
                const float fi = ((float)Xc - X00f) * dXrf * invR2 + ((float)Yr - Y00f) * dYrf * invR2;
                const int ilo = max(0, (int)ceilf(fi - wI)), ihi = min(ns - 1, (int)floorf(fi + wI));
                T gl = T(0), gm = T(0);
                for (int i = ilo; i <= ihi; ++i) {
                    const int c = scnt[i];
                    if (c == 0) continue;
                    int k = max(0, (int)floorf((sYf[i] - (float)(Yr + 1)) * invdY) - 1);
                    for (; k < c; ++k) {
                        const int idx = SBi[k * nth + i];
                        const int iy0 = (idx >> 16) - 1;
                        if (iy0 > Yr) continue;
                        if (iy0 < Yr - 1) break;
                        const int dx = Xc - ((idx & 0xffff) - 1);
                        if (dx != 0 && dx != 1) continue;
                        const T2 axy = SBa[k * nth + i];
                        const T2 gg = SBg[k * nth + i];
                        const T wx = dx == 0 ? T(1) - axy.x : axy.x;
                        const T wy = iy0 == Yr ? T(1) - axy.y : axy.y;
                        const T wgt = wx * wy;
                        gl += wgt * gg.x;
                        gm += wgt * gg.y;
                    }
                }
                if (ck > 0 && Yr == row_hi + 1) {
                    gl += carry_rd[Xc].x;
                    gm += carry_rd[Xc].y;
                }
                if (Yr == row_lo && ck < A.nchunks - 1) {
                    carry_wr[Xc] = mk2(gl, gm);
                } else {
                    const int row = vp.flipped ? (n - 1 - Yr) : Yr;
                    gp[(size_t)row * n + Xc] = gl;
                    gp[(size_t)n * n + (size_t)row * n + Xc] = gm;
                }
            }
        }
    }

    if constexpr (MODE == kFwd || MODE == kJvp) {
        const T val = q.val();
        if (active) {
            sval[tid] = val;
            if (MODE == kFwd && A.slot_val) ((T*)A.slot_val)[(size_t)v * A.max_slots + tid] = val;
        }
        __syncthreads();
        T* y = (T*)A.y_out + (size_t)vp.angle * A.n_det + (size_t)vp.bank * A.nb;
        for (int d = tid; d < A.nb; d += nth) {
            const int* ds = A.det_slot + (size_t)(vp.bank * A.nb + d) * A.n_sub;
            T acc = T(0);
            for (int k = 0; k < A.n_sub; ++k) acc += (T)A.w[k] * sval[ds[k]];
            y[d] = h * acc;
        }
    }
}

static size_t walk_smem(int mode, bool f64, int threads, int Yc, int P, int n, int cap) {
    size_t s2 = f64 ? 16 : 8;
    size_t b = s2 * (size_t)(Yc + 1) * P * (mode == kJvp ? 2 : 1) + s2 * threads;
    if (mode == kVjp) b += (2 * s2 + 4) * (size_t)cap * threads + 2 * s2 * n + 8 * (size_t)threads;
    return b;
}

WalkPlan plan_walk(const Geometry& g, int P, int mode, bool f64, size_t budget) {
    WalkPlan pl;
    pl.threads = ((g.max_slots + 31) / 32) * 32;
    int best = 1;
    for (int Yc = 1; Yc <= g.n + 1; ++Yc) {
        int cap = (mode == kVjp) ? (int)(Yc * 1.41421357 / g.h) + 3 : 0;
        if (walk_smem(mode, f64, pl.threads, Yc, P, g.n, cap) <= budget) best = Yc;
        else break;
    }
    pl.Yc = best;
    pl.nchunks = (g.n + 1 + best - 1) / best;
    pl.sb_cap = (mode == kVjp) ? (int)(best * 1.41421357 / g.h) + 3 : 0;
    pl.smem = walk_smem(mode, f64, pl.threads, best, P, g.n, pl.sb_cap);
    return pl;
}

template <typename T, bool K, int M>
static cudaError_t launch_one(const WalkPlan& pl, const WalkArgs& a, int n_views, cudaStream_t st) {
    auto kern = walk_kernel<T, K, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<n_views, pl.threads, pl.smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_walk(int mode, int precision, const WalkPlan& pl, const WalkArgs& a, int n_views,
                        cudaStream_t st) {
    if (n_views <= 0) return cudaSuccess;
#define PGET_L(T, K)                                                           \
    switch (mode) {                                                            \
        case kFwd: return launch_one<T, K, kFwd>(pl, a, n_views, st);          \
        case kJvp: return launch_one<T, K, kJvp>(pl, a, n_views, st);          \
        default: return launch_one<T, K, kVjp>(pl, a, n_views, st);            \
    }
    if (precision == PGET_F64) {
        PGET_L(double, false)
    } else if (precision == PGET_F32) {
        PGET_L(float, false)
    } else {
        PGET_L(float, true)
    }
#undef PGET_L
}

}  // namespace pget
