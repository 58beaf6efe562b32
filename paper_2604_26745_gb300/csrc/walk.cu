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
//     ray total (from the forward pass) minus the detector-side suffix.
// With the depth factors of Eq. (5) (DEPTH): e_j = w_j exp(-c_j E_j) in all three, dE_j
// enters the JVP as c_j dE_j, and the adjoint prefix sums c_l lambda_l e_l (the forward
// then stores that c-weighted total for the adjoint).
//
// Scatter-free adjoint.  A sample touches the four pixels of its bilinear cell: columns
// ix0, ix0+1 of rows iy0, iy0+1.  Every ray crosses a pixel row with at most three
// samples whose cells touch that row (the canonical frame guarantees |dX| <= |dY| per
// step), and those cells lie within four consecutive columns.  While walking, the
// thread that owns a ray accumulates, for each row of the current chunk, its exact
// bilinear contributions into a private 4-column stencil in shared memory (origin c0 per
// (ray, row)).  After the chunk every pixel GATHERS from the stencils of the few rays
// whose footprint covers it: no atomics, no write conflicts, deterministic order.  Rows
// shared by consecutive chunks are completed through a carried pixel row; each view
// writes its own partial image, reduce_views sums them in a fixed order.
//
// Phase buffers (kVjpP, for slot lattices that need at most kMaxPhases phases).  The rays
// of slots t and t + K of a view never touch the same pixel when K slot steps, measured
// along a pixel row, span more than the columns a ray's cells cover in two rows
// (adjoint_phases_needed).  Each ray then accumulates straight into the row buffer of its
// phase t mod K, a dense copy of the chunk's rows that no other ray writes at those pixels,
// and every pixel sums its K buffers in phase order: no stencil origins, no candidate
// search, still no atomics and a fixed order.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <utility>

#include "kernels.cuh"

namespace pget {

static std::atomic<long long> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

constexpr short kNoRow = -30000;  // stencil origin of a (ray, row) the ray never touched

// Stencil columns per (ray, row).  The cells touching one row span at most three base
// columns; the float paths step positions in exact 32.32 fixed point so four columns
// always suffice, the double path evaluates positions per sample and keeps one column
// of slack for rounding at exactly 45-degree views.
template <typename T> constexpr int stencil_width() { return sizeof(T) == 8 ? 5 : 4; }

// two neighbouring shared-memory elements from a 16-byte aligned address (one vector
// load for float pairs)
__device__ __forceinline__ void ld_pair(const float2* p, float2* a, float2* b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    *a = make_float2(v.x, v.y);
    *b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2* a, double2* b) {
    *a = p[0];
    *b = p[1];
}
__device__ __forceinline__ void zero_pair(float2* p) { *reinterpret_cast<float4*>(p) = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero_pair(double2* p) { p[0] = p[1] = make_double2(0.0, 0.0); }

// ---- chunk staging: TMA bulk copies (cp.async.bulk) completing on an mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(unsigned long long* mb, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}
// make the initialised barriers visible to the async proxy (the copy engine)
__device__ __forceinline__ void mb_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// order earlier generic-proxy accesses of shared memory before later async-proxy writes
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mb_expect_tx(unsigned long long* mb, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mb))
                 : "memory");
}
__device__ __forceinline__ bool mb_try_wait(unsigned long long* mb, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(mb)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for a phase of a chunk barrier, for at most limit_ns of device time (globaltimer).
// Returns false when the limit ran out: the caller records the error and stops issuing
// copies, so a lost copy never hangs the GPU.
__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mb_wait(unsigned long long* mb, unsigned parity, long long limit_ns) {
    if (mb_try_wait(mb, parity)) return true;
    const unsigned long long t0 = gtimer_ns();
    while (!mb_try_wait(mb, parity))
        if (gtimer_ns() - t0 > (unsigned long long)limit_ns) return false;
    return true;
}

// Copy canonical rows [row_lo, row_lo + nrows) of a padded layout into a shared-memory
// chunk (row pitch Ps): one bulk copy per row of P elements, issued by the lanes of one
// warp in parallel (lane k takes rows k, k + 32, ...).  Row bytes, source and destination
// offsets are multiples of 16 (P and Ps even).
template <typename T2>
__device__ __forceinline__ void issue_rows(T2* dst, const T2* src, int P, int Ps, int n, int flipped, int row_lo,
                                           int nrows, unsigned long long* mb, int lane) {
    const unsigned bytes = (unsigned)(P * sizeof(T2));
    for (int rr = lane; rr < nrows; rr += 32) {
        const int r = row_lo + rr;
        const int gr = (flipped ? (n - 1 - r) : r) + 1;
        bulk_g2s(dst + (size_t)rr * Ps, src + (size_t)gr * P, bytes, mb);
    }
}

// Copy canonical rows [row_lo, row_lo + nrows) of a padded layout into shared memory with
// plain loads: one warp per row, 16-byte vectors (P is even, so a row of float2 is a whole
// number of 16-byte vectors; a double2 is one vector).
template <typename T2>
__device__ __forceinline__ void stage_rows(T2* __restrict__ dst, const T2* __restrict__ src, int P, int Ps,
                                           int n, int flipped, int row_lo, int nrows) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int per = 16 / sizeof(T2);  // elements per 16-byte vector
    const int nvec = P / per;
    for (int rr = warp; rr < nrows; rr += nw) {
        const int r = row_lo + rr;
        const int gr = (flipped ? (n - 1 - r) : r) + 1;
        const float4* s = reinterpret_cast<const float4*>(src + (size_t)gr * P);
        float4* d = reinterpret_cast<float4*>(dst + (size_t)rr * Ps);
        for (int c = lane; c < nvec; c += 32) d[c] = s[c];
    }
}

// rows of chunk ck: base rows row_hi down to row_lo, staged rows row_lo .. row_hi + 1
__device__ __forceinline__ void chunk_rows(int n, int Yc, int ck, int* row_hi, int* row_lo, int* nrows) {
    *row_hi = n - 1 - ck * Yc;
    *row_lo = max(-1, *row_hi - Yc + 1);
    *nrows = *row_hi - *row_lo + 2;
}

// MAXT: the largest block the instantiation launches with.  The kWalkThreads
// instantiation may use 72 registers per thread (measured 4-12 % faster than 64 at 3 CTAs
// of 288 threads per SM); it runs when the view has at most kWalkThreads rays and the
// extra registers leave as many CTAs resident per SM (see walk_choice).  Otherwise the
// kMaxSlots instantiation runs, 64 registers, so that 1024 threads fit.
template <typename T, bool KAHAN, int MODE, bool DEPTH, int MAXT>
__global__ void __maxnreg__(MAXT <= kWalkThreads ? 72 : 64) walk_kernel(WalkArgs A) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char sm[];
    if (A.stop && *A.stop) return;
    // batched launches: item blockIdx.y of a batch of independent images (same geometry),
    // its arrays at the item strides (bytes); 0 strides for a single item
    const long long item = blockIdx.y;
    const unsigned char* const u_img0 = (const unsigned char*)A.u_img[0] + item * A.s_img;
    const unsigned char* const u_img1 = (const unsigned char*)A.u_img[1] + item * A.s_img;
    const unsigned char* const p_img0 = (const unsigned char*)A.p_img[0] + item * A.s_img;
    const unsigned char* const p_img1 = (const unsigned char*)A.p_img[1] + item * A.s_img;
    unsigned char* const y_out = (unsigned char*)A.y_out + item * A.s_sino;
    const unsigned char* const r_in = (const unsigned char*)A.r_in + item * A.s_sino;
    unsigned char* const slot_val = A.slot_val ? (unsigned char*)A.slot_val + item * A.s_slot : nullptr;
    unsigned char* const gpart = (unsigned char*)A.gpart + item * A.s_part;
    const int n = A.n, P = A.P, Ps = A.Ps, Yc = A.Yc, tid = threadIdx.x;
    const int nth = A.nst;  // stencil plane stride (>= blockDim.x)
    const T h = (T)A.h;
    constexpr int SW = stencil_width<T>();

    // row buffers: the forward and the JVP double-buffer their chunks, which arrive by TMA
    // bulk copies (the next chunk is copied while the current one is walked); the adjoint
    // stages its single buffer with plain loads of all warps between its chunks (measured
    // faster there: its short chunks alternate walk and gather phases)
    constexpr bool VJP = MODE == kVjp || MODE == kVjpP;  // adjoint: stencils, or phase buffers (PH)
    constexpr bool PH = MODE == kVjpP;
    constexpr int NB = VJP ? 1 : 2;
    constexpr bool TMA = !VJP;
    const size_t rbytes = sizeof(T2) * (size_t)(Yc + 1) * Ps;  // one staged image chunk
    size_t off = 0;
    T2* const cu0 = (T2*)sm;  // buffer 0: (lambda, mu) [, (dlambda, dmu)]; buffer 1 follows
    off += NB * rbytes * (MODE == kJvp ? 2 : 1);
    T* sval = (T*)(sm + off);  // forward / JVP: ray totals
    if constexpr (!VJP) off += sizeof(T2) * (size_t)nth;  // T2-sized: keeps alignment
    T2 *ST = nullptr, *carry0 = nullptr, *carry1 = nullptr, *PB = nullptr;
    short* C0 = nullptr;
    if constexpr (PH) {
        PB = (T2*)(sm + off);  // [phase][row][column + 2]: 16-byte aligned rows (Pb, phs even)
        off += sizeof(T2) * (size_t)A.nph * A.phs;
        carry0 = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)n;
        carry1 = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)n;
    }
    if constexpr (MODE == kVjp) {
        ST = (T2*)(sm + off);  // [(row * SW + k) * nth + ray]
        off += sizeof(T2) * (size_t)(Yc + 1) * SW * nth;
        carry0 = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)n;
        carry1 = (T2*)(sm + off);
        off += sizeof(T2) * (size_t)n;
        C0 = (short*)(sm + off);  // [row * nth + ray]
        off += sizeof(short) * (size_t)(Yc + 1) * nth;
    }
    off = (off + 7) / 8 * 8;
    unsigned long long* mb = (unsigned long long*)(sm + off);  // one barrier per row buffer
    int* s_abort = (int*)(mb + NB);  // set when a copy wait ran out: no further copies
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) mb_init(&mb[b], 1);
        mb_init_fence();
        *s_abort = 0;
    }
    __syncthreads();
    unsigned phase = 0;    // bit b: parity of the next completed phase of buffer b
    unsigned pend = 0;     // bit b: a copy into buffer b was issued and not yet waited for
    bool aborted = false;  // uniform copy of *s_abort, refreshed after barriers
    const long long wait_ns = A.wait_ns > 0 ? A.wait_ns : 1000000000LL;

    // the views of this CTA: one view, or (VJP) a group of views sharing the canonical
    // orientation whose adjoint images are summed into the group's partial image
    // adjoint with phase buffers: the buffer of this thread's ray (slot tid) is tid mod nph
    const int ph_off = PH ? (tid % A.nph) * A.phs : 0;
    const int g = A.cta_order ? A.cta_order[blockIdx.x] : (int)blockIdx.x;
    const int gb = A.group_off ? A.group_off[g] : g;
    const int ge = A.group_off ? A.group_off[g + 1] : g + 1;
    for (int gi = gb; gi < ge; ++gi) {
    const int v = A.group_view ? A.group_view[gi] : gi;
    const bool first_view = gi == gb;
    const ViewDev vp = A.views[v];
    const int ns = vp.n_slots;
    const bool active = tid < ns;
    const T2* ug = (const T2*)(vp.transposed ? u_img1 : u_img0);
    const T2* pg = (MODE == kJvp) ? (const T2*)(vp.transposed ? p_img1 : p_img0) : nullptr;

    const int2 jr = active ? A.clip[(size_t)v * A.max_slots + tid] : make_int2(0, -1);
    const int jlo = jr.x;
    int j = jr.y;
    Pos<T> pos;
    pos.init(vp, active ? tid : 0, j);
    Acc<T, KAHAN> S, q, dS, qc;  // qc: forward with depth factors, sum c_j w_j lambda_j exp(-c_j E_j)
    S.init();
    q.init();
    dS.init();
    qc.init();
    const T2* dtab = (const T2*)A.depth;
    (void)dtab;
    T rho = T(0), Utot = T(0);
    if constexpr (VJP) {
        if (active) {
            const int q0 = A.src_off[vp.bank * A.max_slots + tid];
            const int q1 = A.src_off[vp.bank * A.max_slots + tid + 1];
            const T* r = (const T*)r_in + (size_t)vp.angle * A.n_det;
            const T* sw = (const T*)A.src_w;
            T acc = T(0);
            for (int e = q0; e < q1; ++e) acc += sw[e] * r[A.src_det[e]];
            rho = acc;
            Utot = ((const T*)slot_val)[(size_t)v * A.max_slots + tid];
        }
    }
    // stencil origin offset: walking down, X moves by -dXs per step; the first sample
    // touching a row then has the largest (dXs > 0) or smallest (dXs < 0) base column
    const int base = vp.dXs > 0 ? SW - 2 : 0;
    int cur_row = INT_MIN;
    int c0_lo = 0, c0_hi = 0;
    // candidate rays of a pixel (float bounds; the stencil origin decides exactly)
    const float X00f = (float)vp.X00d, Y00f = (float)vp.Y00d;
    const float dXrf = (float)vp.dXrd, dYrf = (float)vp.dYrd;
    const float invR2 = 1.0f / (dXrf * dXrf + dYrf * dYrf);
    const float wI = (fabsf(dXrf) + fabsf(dYrf)) * invR2 + 0.01f;
    const float inv_np = 1.0f / (float)((n + 1) / 2);  // pixel pairs per row (gather)

    // copy of chunk ck into buffer b, issued by warp 0: lane 0 announces the bytes on the
    // buffer's barrier, then every lane issues its rows
    auto issue = [&](int ck, int b) {
        int rh, rl, nr;
        chunk_rows(n, Yc, ck, &rh, &rl, &nr);
        if (tid == 0) {
            proxy_fence();
            mb_expect_tx(&mb[b], (unsigned)(nr * P * sizeof(T2)) * (MODE == kJvp ? 2u : 1u) +
                                     (ck == 0 ? (unsigned)A.tx_extra : 0u));
        }
        __syncwarp();
        T2* dst = (T2*)((unsigned char*)cu0 + (size_t)b * rbytes * (MODE == kJvp ? 2 : 1));
        issue_rows(dst, ug, P, Ps, n, vp.flipped, rl, nr, &mb[b], tid);
        if constexpr (MODE == kJvp)
            issue_rows((T2*)((unsigned char*)dst + rbytes), pg, P, Ps, n, vp.flipped, rl, nr, &mb[b], tid);
    };
    if (TMA && !aborted) {  // the buffers are free: the previous view ended with a barrier
        if (tid < 32) issue(0, 0);
        pend |= 1u;
    }

    for (int ck = 0; ck < A.nchunks; ++ck) {
        int row_hi, row_lo, nrows;
        chunk_rows(n, Yc, ck, &row_hi, &row_lo, &nrows);
        const int b = NB == 2 ? (ck & 1) : 0;
        if constexpr (NB == 2)  // buffer b ^ 1 was released by the barrier ending chunk ck - 1
            if (!aborted && ck + 1 < A.nchunks) {
                if (tid < 32) issue(ck + 1, b ^ 1);
                pend |= 1u << (b ^ 1);
            }
        // adjoint: stencil columns cover the window of rays with samples in this chunk
        int wa = 0, wn = 0, ts = 0;
        bool in_win = false;
        if constexpr (MODE == kVjp) {
            const int2 wv = A.win ? A.win[(size_t)v * A.nchunks + ck] : make_int2(0, ns);
            wa = wv.x;
            wn = wv.y;
            ts = tid - wa;
            in_win = (unsigned)ts < (unsigned)wn;
            __syncthreads();  // the gather of chunk ck - 1 has read every stencil
            // column ts belongs to the ray of thread wa + ts: the thread that writes it during
            // the walk also clears it, so no barrier is needed between the two
            if (in_win)
                for (int rr = 0; rr < nrows; ++rr) {
                    C0[rr * nth + ts] = kNoRow;
#pragma unroll
                    for (int k = 0; k < SW; ++k) ST[(rr * SW + k) * nth + ts] = mk2(T(0), T(0));
                }
            cur_row = INT_MIN;  // the stencil rows of this chunk start empty
        }
        if constexpr (PH) {
            // the view's first chunk finds the buffers zeroed here (the previous view ended
            // with a barrier); every later chunk finds them zeroed by the gather before it
            if (ck == 0) {
                const int per_phase = (Yc + 1) * A.Pb * (int)sizeof(T2) / 16;
                for (int k = 0; k < A.nph; ++k) {
                    float4* d = reinterpret_cast<float4*>(PB + (size_t)k * A.phs);
                    for (int e = tid; e < per_phase; e += blockDim.x) d[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        if constexpr (TMA) {
            if (pend & (1u << b)) {  // after an abort the buffer holds stale rows: results are void
                if (!mb_wait(&mb[b], (phase >> b) & 1u, wait_ns)) {
                    atomicOr(A.err, 4);
                    *s_abort = 1;
                }
                phase ^= 1u << b;
                pend &= ~(1u << b);
            }
        } else if (!PH || ck == 0) {  // the phase-buffer adjoint stages later chunks after each gather
            stage_rows(cu0, ug, P, Ps, n, vp.flipped, row_lo, nrows);
            __syncthreads();
        }
        const T2* cu = (const T2*)((const unsigned char*)cu0 + (size_t)b * rbytes * (MODE == kJvp ? 2 : 1));
        const T2* cp = (const T2*)((const unsigned char*)cu + rbytes);  // JVP only
        (void)cp;
        if (active) {
            while (j >= jlo) {
                const int iy0 = pos.iy();
                if (iy0 < row_lo) break;
                const int ix0 = pos.ix();
                if (iy0 <= row_hi && ix0 >= -1 && ix0 <= n - 1) {
                    const T ax = pos.ax(), ay = pos.ay();
                    const int o = (iy0 - row_lo) * Ps + ix0 + 1;
                    const T2 a00 = cu[o], a10 = cu[o + 1], a01 = cu[o + Ps], a11 = cu[o + Ps + 1];
                    const T w11 = ax * ay, w10 = ax - w11, w01 = ay - w11;
                    const T w00 = (T(1) - ax) - w01;
                    const T2 lm = bilerp2(w00, w10, w01, w11, a00, a10, a01, a11);
                    const T l = lm.x, m = lm.y;  // m is mu h log2(e)
                    T dw = T(1), dc = T(1);    // depth factors of sample j
                    if constexpr (DEPTH) {
                        const T2 t = dtab[j];
                        dw = t.x;
                        dc = t.y;
                    }
                    const T at = DEPTH ? exp2_(-(dc * (S.val() + T(0.5) * m))) : exp2_(-(S.val() + T(0.5) * m));
                    if constexpr (MODE == kFwd) {
                        if constexpr (DEPTH) {
                            const T wl = dw * (l * at);
                            q.add(wl);
                            qc.add(dc * wl);
                        } else {
                            q.add(l * at);
                        }
                    } else if constexpr (MODE == kJvp) {
                        const T2 b00 = cp[o], b10 = cp[o + 1], b01 = cp[o + Ps], b11 = cp[o + Ps + 1];
                        const T2 dd = bilerp2(w00, w10, w01, w11, b00, b10, b01, b11);
                        // dE in natural units: ln 2 (dS + dm/2) with dS, dm scaled like m
                        const T dE = T(0.6931471805599453) * (dS.val() + T(0.5) * dd.y);
                        if constexpr (DEPTH) q.add(dw * at * (dd.x - l * (dc * dE)));
                        else q.add(at * (dd.x - l * dE));
                        dS.add(dd.y);
                    } else {
                        const T la = DEPTH ? dw * (l * at) : l * at;  // emission term of sample j
                        const T cla = DEPTH ? dc * la : la;            // its weight in the prefix
                        const T Qh = (Utot - q.val()) - T(0.5) * cla;
                        const T gl = DEPTH ? rho * h * (dw * at) : rho * h * at;
                        const T gm = -rho * h * h * Qh;
                        const int rl = iy0 - row_lo;  // lower row of the cell; upper is rl + 1
                        if constexpr (PH) {
                            // the ray's own phase buffer: no other ray of this phase touches
                            // these cells in this chunk (the plan's phase count guarantees it)
                            T2* pb = PB + ph_off + rl * A.Pb + ix0 + 2;
                            const T2 g2 = mk2(gl, gm);
                            const T2 t0 = pb[0], t1 = pb[1], t2 = pb[A.Pb], t3 = pb[A.Pb + 1];
                            pb[0] = fma2(w00, g2, t0);
                            pb[1] = fma2(w10, g2, t1);
                            pb[A.Pb] = fma2(w01, g2, t2);
                            pb[A.Pb + 1] = fma2(w11, g2, t3);
                        } else {
                            if (iy0 != cur_row && in_win) {  // stencil rows start zeroed (chunk top)
                                if (iy0 + 1 != cur_row) {
                                    c0_hi = ix0 - base;
                                    C0[(rl + 1) * nth + ts] = (short)c0_hi;
                                } else {
                                    c0_hi = c0_lo;
                                }
                                c0_lo = ix0 - base;
                                C0[rl * nth + ts] = (short)c0_lo;
                                cur_row = iy0;
                            }
                            const int ol = ix0 - c0_lo, oh = ix0 - c0_hi;
                            // in_win holds by construction of the windows; never write outside them
                            if ((unsigned)ol <= (unsigned)(SW - 2) && (unsigned)oh <= (unsigned)(SW - 2) && in_win) {
                                T2* pl = ST + (size_t)(rl * SW + ol) * nth + ts;
                                T2* ph = ST + (size_t)((rl + 1) * SW + oh) * nth + ts;
                                const T2 g2 = mk2(gl, gm);
                                const T2 t0 = pl[0], t1 = pl[nth], t2 = ph[0], t3 = ph[nth];
                                pl[0] = fma2(w00, g2, t0);
                                pl[nth] = fma2(w10, g2, t1);
                                ph[0] = fma2(w01, g2, t2);
                                ph[nth] = fma2(w11, g2, t3);
                            } else {
                                atomicOr(A.err, 2);  // geometry bound violated: report, never write out of range
                            }
                        }
                        q.add(cla);
                    }
                    S.add(m);
                }
                --j;
                pos.back();
            }
        }
        __syncthreads();  // every walk of chunk ck is done: its row buffer is free
        if constexpr (TMA) aborted = *s_abort != 0;
        if constexpr (VJP) {
            const int r0 = max(row_lo, 0), r1 = min(row_hi + 1, n - 1);
            T2* carry_rd = (ck & 1) ? carry0 : carry1;
            T2* carry_wr = (ck & 1) ? carry1 : carry0;
            T* gp = (T*)gpart + (size_t)g * 2 * n * n;
            // every thread gathers two neighbouring pixels (Xa, Xa + 1) of a row.  Stencils:
            // their candidate rays overlap, so one pass over the union loads each ray's
            // stencil origin once; a ray outside one pixel's own window holds zeros at that
            // pixel, and each pixel's sum keeps the ascending order of the rays.  Phase
            // buffers: the pixel's value in each phase (at most one ray of a phase touches
            // it), summed in phase order
            const int npair = (n + 1) / 2;
            const int nout2 = (r1 - r0 + 1) * npair;
            for (int e2 = tid; e2 < nout2; e2 += blockDim.x) {
                const int dy = __float2int_rz(((float)e2 + 0.5f) * inv_np);
                const int Yr = r0 + dy, Xa = 2 * (e2 - dy * npair);
                const int rl = Yr - row_lo;
                T2 acca = mk2(T(0), T(0)), accb = mk2(T(0), T(0));
                if constexpr (PH) {
                    // read and clear: the next chunk's walk finds the entries at zero
                    T2* src = PB + rl * A.Pb + Xa + 2;  // even offset: 16-byte aligned pair
                    // up to four phases loaded before any is cleared, so that the loads
                    // overlap; summed in phase order.  Only in the float 72-register
                    // instantiation: measured 206 -> 196-201 us at 128^2 x 360 x 182 x 5 and
                    // 488 -> 430 us at 256^2, but 3.10 -> 3.34 ms in the 64-register one
                    // (512^2 x 720 x 182 x 9), and spills in double
                    constexpr int G = (sizeof(T) == 4 && MAXT <= kWalkThreads) ? 4 : 1;
                    for (int k0 = 0; k0 < A.nph; k0 += G) {
                        const int nk = min(G, A.nph - k0);
                        T2 va[G], vb[G];
#pragma unroll
                        for (int k = 0; k < G; ++k)
                            if (k < nk) ld_pair(src + (size_t)(k0 + k) * A.phs, &va[k], &vb[k]);
#pragma unroll
                        for (int k = 0; k < G; ++k)
                            if (k < nk) {
                                zero_pair(src + (size_t)(k0 + k) * A.phs);
                                acca = add2(acca, va[k]);
                                accb = add2(accb, vb[k]);
                            }
                    }
                } else {
                    const float fa = ((float)Xa - X00f) * dXrf * invR2 + ((float)Yr - Y00f) * dYrf * invR2;
                    const float fb = fa + dXrf * invR2;
                    const int ilo = max(0, (int)ceilf(fminf(fa, fb) - wI - wa));
                    const int ihi = min(wn - 1, (int)floorf(fmaxf(fa, fb) + wI - wa));
                    const short* c0r = C0 + rl * nth;
                    const T2* str = ST + (size_t)rl * SW * nth;
                    for (int t = ilo; t <= ihi; ++t) {
                        const int ka = Xa - (int)c0r[t];
                        const T2 va = (unsigned)ka < (unsigned)SW ? str[ka * nth + t] : mk2(T(0), T(0));
                        const T2 vb = (unsigned)(ka + 1) < (unsigned)SW ? str[(ka + 1) * nth + t] : mk2(T(0), T(0));
                        acca = add2(acca, va);
                        accb = add2(accb, vb);
                    }
                }
#pragma unroll
                for (int q2 = 0; q2 < 2; ++q2) {
                    const int Xc = Xa + q2;
                    if (Xc >= n) break;
                    T2 acc = q2 ? accb : acca;
                    if (ck > 0 && Yr == row_hi + 1) acc = add2(acc, carry_rd[Xc]);
                    if (Yr == row_lo && ck < A.nchunks - 1) {
                        carry_wr[Xc] = acc;
                    } else {
                        const int row = vp.flipped ? (n - 1 - Yr) : Yr;
                        T* o0 = gp + (size_t)row * n + Xc;
                        T* o1 = o0 + (size_t)n * n;
                        if (first_view) {
                            *o0 = acc.x;
                            *o1 = acc.y;
                        } else {
                            *o0 += acc.x;
                            *o1 += acc.y;
                        }
                    }
                }
            }
            if constexpr (PH) {
                // entries the walk wrote that no pixel pair read: columns -1 and n of every
                // buffer row, and image row n (first chunk); then the next chunk's rows
                const int K = A.nph;
                for (int e = tid; e < K * nrows * 2; e += blockDim.x) {
                    const int k = e / (nrows * 2), rem = e - k * (nrows * 2);
                    PB[(size_t)k * A.phs + (rem >> 1) * A.Pb + ((rem & 1) ? n + 2 : 1)] = mk2(T(0), T(0));
                }
                if (row_hi + 1 == n)
                    for (int e = tid; e < K * (n + 2); e += blockDim.x) {
                        const int k = e / (n + 2), c = e - k * (n + 2);
                        PB[(size_t)k * A.phs + (n - row_lo) * A.Pb + 1 + c] = mk2(T(0), T(0));
                    }
                if (ck + 1 < A.nchunks) {
                    int nh, nl, nr;
                    chunk_rows(n, Yc, ck + 1, &nh, &nl, &nr);
                    stage_rows(cu0, ug, P, Ps, n, vp.flipped, nl, nr);
                }
                __syncthreads();  // buffers back at zero, the next chunk staged
            }
        }
    }

    if constexpr (MODE == kFwd || MODE == kJvp) {
        const T val = q.val();
        if (active) {
            sval[tid] = val;
            // the adjoint's ray total: with depth factors the c-weighted one
            if (MODE == kFwd && slot_val) ((T*)slot_val)[(size_t)v * A.max_slots + tid] = DEPTH ? qc.val() : val;
        }
        __syncthreads();
        T* y = (T*)y_out + (size_t)vp.angle * A.n_det + (size_t)vp.bank * A.nb;
        const T* wk = (const T*)A.w;
        for (int d = tid; d < A.nb; d += blockDim.x) {
            const int* ds = A.det_slot + (size_t)(vp.bank * A.nb + d) * A.n_sub;
            T acc = T(0);
            for (int k = 0; k < A.n_sub; ++k) acc += wk[k] * sval[ds[k]];
            y[d] = h * acc;
        }
    }
    __syncthreads();  // the next view of the group reuses shared memory
    }

}

// shared-memory row pitch of a staged chunk (a skew against bank conflicts between lanes
// sampling two neighbouring rows)
static int smem_pitch(int P, bool f64) {
#ifdef PGET_TUNING
    if (const char* e = getenv("PGET_SMEM_SKEW")) {  // sweep: extra elements per row (even)
        const int k = atoi(e);
        return P + (k > 0 ? (k + 1) / 2 * 2 : 0);
    }
#endif
    // measured best of skews 0..14 at 128 x 128 (forward and JVP): P + 4.  From 256 x 256
    // up (float) a pitch on a multiple of 16 elements measured faster: at 256^2 x 360 x
    // 182 x 5 the JVP 200 -> 171 us and the adjoint 430 -> 424 us, at 512^2 x 720 x 182 x 9
    // the JVP 1.25 -> 1.21 ms, the adjoint 3.10 -> 3.07 ms, the forward 730 -> 722 us; at
    // 192^2 and 128^2 it was slower (adjoint 355 -> 370 us, forward 60 -> 68 us)
    if (!f64 && P >= 258) return (P + 2 + 15) / 16 * 16;
    return P + 4;
}

// stencil plane stride: consecutive planes start 8 words apart modulo the banks, so
// pixels gathering different columns of one ray's stencil do not collide
static int stencil_stride(int threads, bool f64) {
    const int words = f64 ? 4 : 2;
    int s = threads;
    while ((s * words) % 32 != 8) ++s;
    return s;
}

void ray_rows(const Geometry& g, bool f64, std::vector<int2>* rows) {
    const int V = (int)g.views.size(), ms = g.max_slots, n = g.n;
    rows->assign((size_t)V * ms, make_int2(INT_MIN, INT_MIN));
    for (int v = 0; v < V; ++v) {
        const ViewDev& vp = g.views[v];
        for (int i = 0; i < vp.n_slots; ++i) {
            const int jlo = g.clip[((size_t)v * ms + i) * 2], jhi = g.clip[((size_t)v * ms + i) * 2 + 1];
            // base pixel of sample j, exactly as the kernels compute it
            auto cell = [&](int j, long long* ix, long long* iy) {
                if (f64) {
                    const double X0 = std::fma((double)i, vp.dXrd, vp.X00d);
                    const double Y0 = std::fma((double)i, vp.dYrd, vp.Y00d);
                    *ix = (long long)std::floor(std::fma((double)j, vp.dXsd, X0));
                    *iy = (long long)std::floor(std::fma((double)j, vp.dYsd, Y0));
                } else {
                    *ix = (vp.X00 + (long long)i * vp.dXr + (long long)j * vp.dXs) >> 32;
                    *iy = (vp.Y00 + (long long)i * vp.dYr + (long long)j * vp.dYs) >> 32;
                }
            };
            auto valid = [&](int j, long long* iy) {
                long long ix;
                cell(j, &ix, iy);
                return ix >= -1 && ix <= n - 1 && *iy >= -1 && *iy <= n - 1;
            };
            // the valid samples of a straight ray are one contiguous range of j
            long long iy = 0;
            int j1 = jhi;
            while (j1 >= jlo && !valid(j1, &iy)) --j1;
            if (j1 < jlo) continue;
            const int first = (int)iy;
            int j0 = jlo;
            while (!valid(j0, &iy)) ++j0;
            (*rows)[(size_t)v * ms + i] = make_int2(first, (int)iy);
        }
    }
}

// Ray windows of a chunk height: per (view, chunk) the first slot and the number of slots
// spanning every ray with a valid sample in the chunk.  Returns the widest window.
static int chunk_windows(const Geometry& g, const std::vector<int2>& rows, int Yc, int nchunks,
                         std::vector<int2>* win) {
    const int V = (int)g.views.size(), ms = g.max_slots, n = g.n;
    if (win) win->assign((size_t)V * nchunks, make_int2(0, 0));
    std::vector<int> lo(nchunks), hi(nchunks);
    int widest = 0;
    for (int v = 0; v < V; ++v) {
        std::fill(lo.begin(), lo.end(), INT_MAX);
        std::fill(hi.begin(), hi.end(), -1);
        for (int i = 0; i < g.views[v].n_slots; ++i) {
            const int2 r = rows[(size_t)v * ms + i];
            if (r.x == INT_MIN) continue;
            // rows run from n - 1 (chunk 0) down to -1; r.x >= r.y
            const int k0 = (n - 1 - r.x) / Yc, k1 = (n - 1 - r.y) / Yc;
            for (int k = k0; k <= k1; ++k) {
                lo[k] = std::min(lo[k], i);
                hi[k] = std::max(hi[k], i);
            }
        }
        for (int k = 0; k < nchunks; ++k) {
            if (hi[k] < 0) continue;
            if (win) (*win)[(size_t)v * nchunks + k] = make_int2(lo[k], hi[k] - lo[k] + 1);
            widest = std::max(widest, hi[k] - lo[k] + 1);
        }
    }
    return widest;
}

static size_t walk_smem(int mode, bool f64, int threads, int Yc, int Ps, int nst, int n) {
    size_t s2 = f64 ? 16 : 8;
    const size_t nbuf = mode == kVjp ? 1 : 2;  // row buffers (see the kernel)
    size_t b = nbuf * s2 * (size_t)(Yc + 1) * Ps * (mode == kJvp ? 2 : 1) + (mode == kVjp ? 0 : s2 * nst);
    if (mode == kVjp) b += s2 * (size_t)(Yc + 1) * (f64 ? 5 : 4) * nst + 2 * s2 * n + 2 * (size_t)(Yc + 1) * nst;
    b = (b + 7) / 8 * 8 + 8 * nbuf + 8;  // chunk barriers and the abort flag
    (void)threads;
    return (b + 15) / 16 * 16;
}

// Phases of the adjoint's row buffers.  In a view's canonical frame the lines of slots t
// and t + K lie K sigma_h apart horizontally, sigma_h = |dXr - dYr dXs / dYs| (the slot
// step projected along the rays onto a row).  The samples whose cells touch one pixel row
// have Y in [row - 1, row + 1), so their X span is below 2 s (s = |dXs / dYs| <= 1), and
// the columns they write lie in [floor(x_min), floor(x_max) + 1].  K sigma_h >= 2 s + 2
// then keeps the columns of two rays of one phase apart in every row: each phase buffer
// is written by one ray per pixel.  0.05 px of margin covers the rounding of positions.
// Returns 0 when no view allows it (a zero slot step).
int adjoint_phases_needed(const Geometry& g) {
    double need = 1.0;
    for (const ViewDev& v : g.views) {
        const double s = std::fabs(v.dXsd / v.dYsd);
        const double sh = std::fabs(v.dXrd - v.dYrd * v.dXsd / v.dYsd);
        if (!(sh > 1e-9) || !std::isfinite(s)) return 0;
        need = std::max(need, (2.0 * s + 2.05) / sh);
    }
    return need > 1e6 ? 0 : (int)std::ceil(need);
}

// stride between phase buffers of (Yc + 1) rows of pitch Pb: even (16-byte aligned
// buffers) and `bank` words past a multiple of the 32 banks (rounded down to what an even
// stride reaches: a multiple of 2 words per element)
static int phase_stride(int Yc, int Pb, bool f64, int bank) {
    const int words = f64 ? 4 : 2;
    const int target = (bank % 32) / (2 * words) * (2 * words);
    int s = (Yc + 1) * Pb;
    s += s & 1;
    while ((s * words) % 32 != target) s += 2;
    return s;
}

// shared memory of the adjoint with phase buffers: the staged chunk, nph buffers, the two
// carried rows, the barrier and the abort flag
static size_t walk_smem_phases(bool f64, int Yc, int Ps, int nph, int Pb, int n, int bank) {
    const size_t s2 = f64 ? 16 : 8;
    size_t b = s2 * (size_t)(Yc + 1) * Ps + s2 * (size_t)nph * phase_stride(Yc, Pb, f64, bank) + 2 * s2 * n;
    b = (b + 7) / 8 * 8 + 8 + 8;
    return (b + 15) / 16 * 16;
}

// Samples of a few views, in the walk's order, split by chunk: [view][chunk][slot] lists of
// (column, buffer row), for the bank model below.  Positions as in ray_rows (double).
using ChunkSamples = std::vector<std::vector<std::vector<int2>>>;
static std::vector<ChunkSamples> sample_views(const Geometry& g, int Yc, int nviews) {
    const int V = (int)g.views.size(), n = g.n, ms = g.max_slots;
    const int nch = (n + 1 + Yc - 1) / Yc;
    std::vector<ChunkSamples> out;
    for (int q = 0; q < std::min(V, nviews); ++q) {
        const int v = (int)(((2LL * q + 1) * V) / (2LL * std::min(V, nviews)));
        const ViewDev& vp = g.views[v];
        ChunkSamples cs(nch, std::vector<std::vector<int2>>(vp.n_slots));
        for (int i = 0; i < vp.n_slots; ++i) {
            const int jlo = g.clip[((size_t)v * ms + i) * 2], jhi = g.clip[((size_t)v * ms + i) * 2 + 1];
            const double X0 = vp.X00d + i * vp.dXrd, Y0 = vp.Y00d + i * vp.dYrd;
            for (int j = jhi; j >= jlo; --j) {
                const int ix = (int)std::floor(X0 + j * vp.dXsd), iy = (int)std::floor(Y0 + j * vp.dYsd);
                if (ix < -1 || ix > n - 1 || iy < -1 || iy > n - 1) continue;
                const int ck = (n - 1 - iy) / Yc;
                const int row_lo = std::max(-1, n - 1 - ck * Yc - Yc + 1);
                cs[ck][i].push_back(make_int2(ix, iy - row_lo));
            }
        }
        out.push_back(std::move(cs));
    }
    return out;
}

// Modeled shared-memory wavefronts of the phase buffers' read-modify-writes for one layout:
// the lanes of a warp walk consecutive slots in step (iteration k of a chunk: each lane's
// k-th sample in it), a 64-bit (128-bit) access is served per half-warp, and a half-warp
// takes as many wavefronts as the most distinct elements on one bank.  The layout
// (phase stride modulo the banks, row pitch) decides how the lanes' rows, columns and
// phases spread over the banks; measured at 128^2, 256^2 and 512^2 the model ranks the
// layouts as their adjoint times do.
static long long phase_layout_cost(const std::vector<ChunkSamples>& vs, int K, int Pb, int phs, bool f64) {
    const int words = f64 ? 4 : 2;
    long long total = 0;
    for (const ChunkSamples& cs : vs)
        for (const auto& ch : cs)
            for (size_t w0 = 0; w0 < ch.size(); w0 += 32) {
                size_t L = 0;
                for (size_t s = w0; s < std::min(ch.size(), w0 + 32); ++s) L = std::max(L, ch[s].size());
                for (size_t k = 0; k < L; ++k)
                    for (size_t h = w0; h < std::min(ch.size(), w0 + 32); h += 16) {
                        int cnt[32] = {0};
                        for (size_t s = h; s < std::min(ch.size(), h + 16); ++s) {
                            if (k >= ch[s].size()) continue;
                            const long long e = (long long)(s % K) * phs + (long long)ch[s][k].y * Pb + ch[s][k].x + 2;
                            for (int wd = 0; wd < words; ++wd) ++cnt[(int)((e * words + wd) & 31)];
                        }
                        total += *std::max_element(cnt, cnt + 32);
                    }
            }
    return total;
}

// Most phases the adjoint takes phase buffers with: the gather reads every phase per pixel,
// so finer slot lattices keep the per-ray stencils.  Measured (adjoint alone, FP32 + Kahan
// unless stated, phase buffers in the layout the bank model picks vs stencils), K phases:
// 512^2 x 720 x 182 x 9 (K 2) 3.14 vs 4.97 ms; 256^2 x 360 x 182 x 5 (3) 496 vs 547 us;
// 64^2 x 90 x 91 x 1 FP64 (3) 213 vs 259 us; 192^2 x 360 x 182 x 7 (4) 449 vs 559 us;
// 128^2 x 360 x 182 x 5 (5) 210 vs 229 us; 96^2 x 360 x 182 x 5 (6) 150 vs 180 us;
// 128^2 x 360 x 182 x 7 (6) 263 vs 348 us; 128^2 x 360 x 182 x 9 (8) 284 vs 454 us.  A
// -DPGET_TUNING build keeps the stencils when PGET_VJP_DESIGN=stencil.
constexpr int kMaxPhases = 16;


WalkPlan plan_walk(const Geometry& g, int P, int mode, bool f64, size_t budget, const std::vector<int2>* rows) {
    WalkPlan pl;
    pl.threads = ((g.max_slots + 31) / 32) * 32;
    pl.Ps = smem_pitch(P, f64);
    if (mode == kVjp && rows) {
        // tallest chunk whose stencils (as wide as the widest ray window) fit the budget;
        // the window widens with the chunk height, so the fit is monotone in Yc
        auto fits = [&](int Yc, int* nst) {
            const int nch = (g.n + 1 + Yc - 1) / Yc;
            const int W = std::max(1, chunk_windows(g, *rows, Yc, nch, nullptr));
            *nst = stencil_stride(W, f64);
            return walk_smem(mode, f64, pl.threads, Yc, pl.Ps, *nst, g.n) <= budget;
        };
        int lo = 1, hi = g.n + 1, nst = 0;
        while (lo < hi) {  // largest Yc in [1, n + 1] that fits (Yc = 1 if none does)
            const int mid = (lo + hi + 1) / 2;
            if (fits(mid, &nst)) lo = mid;
            else hi = mid - 1;
        }
        fits(lo, &nst);
        // phase buffers instead, when the slot lattice needs few phases and the buffers
        // leave chunks at least as tall as the stencils do
        const int K = adjoint_phases_needed(g);
        int kmax = kMaxPhases;
#ifdef PGET_TUNING
        if (const char* d = getenv("PGET_VJP_DESIGN"))
            if (std::string(d) == "stencil") kmax = 0;
#endif
        const bool phases = K > 0 && K <= kmax;
        if (phases) {
            // the tallest chunk the buffers allow; among the layouts that keep it, the one the
            // bank model rates best (pitch pads 0, 2, 4 elements; phase strides at every bank
            // offset an even stride reaches), ties to the smaller pad and offset
            const int Pb0 = (g.n + 4) / 2 * 2;  // columns -1 .. n at index column + 2, even pitch
            const int step = f64 ? 8 : 4;
            int pads[3] = {0, 2, 4}, npad = 3, banks0 = 0, banks1 = 32 - step;
#ifdef PGET_TUNING
            if (const char* e = getenv("PGET_PHASE_PITCH_PAD")) pads[0] = std::max(0, atoi(e)) / 2 * 2, npad = 1;
            if (const char* e = getenv("PGET_PHASE_BANK")) banks0 = banks1 = std::max(0, atoi(e)) % 32 / step * step;
#endif
            auto fit = [&](int Pb, int bank) {
                int Y = 0;
                for (int Yc = 1; Yc <= g.n + 1; ++Yc) {
                    if (walk_smem_phases(f64, Yc, pl.Ps, K, Pb, g.n, bank) <= budget) Y = Yc;
                    else break;
                }
                return Y;
            };
            int Ymax = 0;
            for (int a = 0; a < npad; ++a)
                for (int bk = banks0; bk <= banks1; bk += step) Ymax = std::max(Ymax, fit(Pb0 + pads[a], bk));
            if (Ymax >= std::max(2, lo)) {
                // views spread over the angles: 16 up to 128^2 (with 6 the model missed the best
                // layout there by 1 %), fewer on large grids, whose plans would otherwise take
                // seconds (the model's cost grows with the samples per view)
                const std::vector<ChunkSamples> vs = sample_views(g, Ymax, g.n <= 128 ? 16 : g.n <= 256 ? 4 : 2);
                long long best = -1;
                int bPb = Pb0, bbank = 0;
                for (int a = 0; a < npad; ++a)
                    for (int bk = banks0; bk <= banks1; bk += step) {
                        const int Pb = Pb0 + pads[a];
                        if (fit(Pb, bk) != Ymax) continue;
                        const long long c = phase_layout_cost(vs, K, Pb, phase_stride(Ymax, Pb, f64, bk), f64);
                        if (best < 0 || c < best) best = c, bPb = Pb, bbank = bk;
                    }
#ifdef PGET_TUNING
                if (getenv("PGET_PLAN_VERBOSE"))
                    fprintf(stderr, "adjoint phases %d: rows %d, pitch %d (pad %d), bank %d, modeled %lld\n", K, Ymax,
                            bPb, bPb - Pb0, bbank, best);
#endif
                pl.Yc = Ymax;
                pl.nchunks = (g.n + 1 + Ymax - 1) / Ymax;
                pl.nph = K;
                pl.Pb = bPb;
                pl.phs = phase_stride(Ymax, bPb, f64, bbank);
                pl.nst = pl.threads;
                pl.sb_cap = 0;
                pl.smem = walk_smem_phases(f64, Ymax, pl.Ps, K, bPb, g.n, bbank);
                return pl;
            }
        }
        pl.Yc = lo;
        pl.nchunks = (g.n + 1 + lo - 1) / lo;
        pl.nst = nst;
        pl.sb_cap = 0;
        pl.smem = walk_smem(mode, f64, pl.threads, lo, pl.Ps, nst, g.n);
        chunk_windows(g, *rows, lo, pl.nchunks, &pl.win);
        return pl;
    }
    pl.nst = mode == kVjp ? stencil_stride(pl.threads, f64) : pl.threads;
    int best = 1;
    for (int Yc = 1; Yc <= g.n + 1; ++Yc) {
        if (walk_smem(mode, f64, pl.threads, Yc, pl.Ps, pl.nst, g.n) <= budget) best = Yc;
        else break;
    }
    pl.Yc = best;
    pl.nchunks = (g.n + 1 + best - 1) / best;
    pl.sb_cap = 0;
    pl.smem = walk_smem(mode, f64, pl.threads, best, pl.Ps, pl.nst, g.n);
    return pl;
}

// Devices the per-device caches below cover (ordinals 0 .. kCacheDevices - 1); a launch on a
// higher ordinal is refused with cudaErrorInvalidDevice.
constexpr int kCacheDevices = 64;

static int current_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) d = -1;
    return d;
}

// dynamic shared memory already permitted for each instantiation, per device (the
// attribute is set per device: a launch on another device needs its own call); set
// outside any stream capture (prepare_walk runs before a CUDA graph is captured) and
// guarded, as contexts may be driven from several host threads
template <typename T, bool K, int M, bool D, int X>
static cudaError_t allow_smem_x(size_t bytes) {
    static std::mutex mu;
    static size_t allowed[kCacheDevices] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= kCacheDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (bytes <= allowed[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<T, K, M, D, X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) allowed[dev] = bytes;
    return e;
}
template <typename T, bool K, int M, bool D>
static cudaError_t allow_smem(size_t bytes) {
    cudaError_t e = allow_smem_x<T, K, M, D, kWalkThreads>(bytes);
    return e != cudaSuccess ? e : allow_smem_x<T, K, M, D, kMaxSlots>(bytes);
}

// The instantiation for a plan: the 72-register one when the block fits it and it keeps
// at least as many CTAs resident per SM as the 64-register one (with 480 threads, say,
// 72 registers allow one CTA per SM where 64 allow two).  The occupancy query runs once per
// (device, block, shared memory) and is cached in a fixed table (no heap allocation, so
// the allocation-free entry point can use it): prepare_walk makes it before any stream
// capture.  When the table is full the query runs again on each launch (never expected:
// a process sees a handful of plan shapes).  Needs allow_smem first.
struct ChoiceEntry {
    int dev, threads;
    size_t smem;
    bool wide;
};
constexpr int kChoiceEntries = 256;

template <typename T, bool K, int M, bool D>
static void (*walk_choice(const WalkPlan& pl))(WalkArgs) {
    if (pl.threads > kWalkThreads) return walk_kernel<T, K, M, D, kMaxSlots>;
    static std::mutex mu;
    static ChoiceEntry table[kChoiceEntries];
    static int used = 0;
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < used; ++i)
        if (table[i].dev == dev && table[i].threads == pl.threads && table[i].smem == pl.smem)
            return table[i].wide ? walk_kernel<T, K, M, D, kWalkThreads> : walk_kernel<T, K, M, D, kMaxSlots>;
    int o72 = 0, o64 = 0;
    const bool ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o72, walk_kernel<T, K, M, D, kWalkThreads>,
                                                                  pl.threads, pl.smem) == cudaSuccess &&
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o64, walk_kernel<T, K, M, D, kMaxSlots>,
                                                                  pl.threads, pl.smem) == cudaSuccess;
    if (!ok) cudaGetLastError();  // a failed query is no launch error: the 64-register one runs
    const bool wide = ok && o72 >= o64 && o72 > 0;
    if (used < kChoiceEntries) table[used++] = ChoiceEntry{dev, pl.threads, pl.smem, wide};
    return wide ? walk_kernel<T, K, M, D, kWalkThreads> : walk_kernel<T, K, M, D, kMaxSlots>;
}

template <typename T, bool K, int M, bool D>
static cudaError_t launch_one(const WalkPlan& pl, const WalkArgs& a0, int n_views, cudaStream_t st) {
    cudaError_t e = allow_smem<T, K, M, D>(pl.smem);
    if (e != cudaSuccess) return e;
    auto kern = walk_choice<T, K, M, D>(pl);
    WalkArgs a = a0;
    a.Ps = pl.Ps;
    a.nst = pl.nst;
    a.nph = pl.nph;
    a.Pb = pl.Pb;
    a.phs = pl.phs;
    kern<<<dim3((unsigned)n_views, (unsigned)std::max(1, a.n_items)), pl.threads, pl.smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, bool K, int M>
static int occ_one(const WalkPlan& pl) {
    // without depth tables (sizes optional view groups only)
    if (allow_smem<T, K, M, false>(pl.smem) != cudaSuccess) return 1;
    auto kern = walk_choice<T, K, M, false>(pl);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, pl.threads, pl.smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

int walk_occupancy(int mode, int precision, const WalkPlan& pl) {
#define PGET_O(T, K)                                      \
    switch (mode) {                                       \
        case kFwd: return occ_one<T, K, kFwd>(pl);        \
        case kJvp: return occ_one<T, K, kJvp>(pl);        \
        default: return pl.nph ? occ_one<T, K, kVjpP>(pl) \
                               : occ_one<T, K, kVjp>(pl); \
    }
    if (precision == PGET_F64) {
        PGET_O(double, false)
    } else if (precision == PGET_F32) {
        PGET_O(float, false)
    } else {
        PGET_O(float, true)
    }
#undef PGET_O
}

// shared memory permitted and the register instantiation chosen for both depth variants
template <typename T, bool K, int M>
static cudaError_t prepare_one(const WalkPlan& pl) {
    cudaError_t e = allow_smem<T, K, M, false>(pl.smem);
    if (e == cudaSuccess) e = allow_smem<T, K, M, true>(pl.smem);
    if (e != cudaSuccess) return e;
    walk_choice<T, K, M, false>(pl);
    walk_choice<T, K, M, true>(pl);
    return cudaSuccess;
}

cudaError_t prepare_walk(int mode, int precision, const WalkPlan& pl) {
#define PGET_P(T, K)                                                                             \
    switch (mode) {                                                                              \
        case kFwd: return prepare_one<T, K, kFwd>(pl);                                           \
        case kJvp: return prepare_one<T, K, kJvp>(pl);                                           \
        default: return pl.nph ? prepare_one<T, K, kVjpP>(pl) : prepare_one<T, K, kVjp>(pl);     \
    }
    if (precision == PGET_F64) {
        PGET_P(double, false)
    } else if (precision == PGET_F32) {
        PGET_P(float, false)
    } else {
        PGET_P(float, true)
    }
#undef PGET_P
}

cudaError_t launch_walk(int mode, int precision, const WalkPlan& pl, const WalkArgs& a, int n_views,
                        cudaStream_t st) {
    if (n_views <= 0) return cudaSuccess;
#define PGET_L(T, K)                                                                                  \
    switch (mode) {                                                                                   \
        case kFwd: return a.depth ? launch_one<T, K, kFwd, true>(pl, a, n_views, st)                  \
                                  : launch_one<T, K, kFwd, false>(pl, a, n_views, st);                \
        case kJvp: return a.depth ? launch_one<T, K, kJvp, true>(pl, a, n_views, st)                  \
                                  : launch_one<T, K, kJvp, false>(pl, a, n_views, st);                \
        default:                                                                                      \
            if (pl.nph) return a.depth ? launch_one<T, K, kVjpP, true>(pl, a, n_views, st)           \
                                       : launch_one<T, K, kVjpP, false>(pl, a, n_views, st);         \
            return a.depth ? launch_one<T, K, kVjp, true>(pl, a, n_views, st)                         \
                           : launch_one<T, K, kVjp, false>(pl, a, n_views, st);                       \
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
