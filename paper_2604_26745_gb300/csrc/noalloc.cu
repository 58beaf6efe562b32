// noalloc.cu -- pget_forward_noalloc: the forward projector for callers that must not
// allocate memory.
//
// Why it exists.  The regular entry points keep their scratch (packed image layouts,
// geometry tables) in a pget_ctx workspace obtained with cudaMalloc.  Some callers cannot
// do that: code running where the caching allocator of another framework owns the device
// memory and no other allocation is tolerated, code inside an allocation-free real-time
// section, or a process whose memory budget is fixed up front.  For them this file keeps
// all scratch of one forward projection in a single fixed array in device memory that
// exists for as long as the library is loaded.
//
// Rules of use (also in include/pget.h):
//   - scratch is kNoAllocScratchBytes (8 MiB) per device that loads the library; a
//     geometry needing more is rejected with PGET_ENOMEM before any work is queued;
//   - the first call on a device looks up the array's device address (cudaGetSymbolAddress
//     with that device current) and caches it; make that first call before any stream
//     capture;
//   - every call uses the same array and overwrites it; calls that overlap on the GPU
//     (different streams, or several host threads) race and give wrong results;
//   - the host side of every call (building the geometry tables in one process-wide
//     staging buffer and copying them to the device) runs under one process-wide mutex,
//     so calls from several host threads, on one device or several, never mix their
//     tables; the device-side race above remains for calls on one device;
//   - the call refuses to run while its stream is being captured into a CUDA graph
//     (PGET_EINVAL): the table copy reads the shared staging buffer when it runs;
//   - the call waits for its forward projection and reads the kernel's error word: a
//     chunk copy that did not arrive in time returns PGET_ETIMEOUT, never a void result;
//   - the call allocates no device or host memory; errors are reported by the returned
//     status only (pget_last_error is not updated, because storing a message may allocate).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <utility>

#include "kernels.cuh"
#include "pget_internal.cuh"
#include "vec.cuh"

namespace pget {

constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr int kNoAllocMaxDevices = 64;

// the scratch array; device code could name it directly, host code only through the
// address cudaGetSymbolAddress returns (the host-side symbol is a stand-in, not a
// device address)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// host staging for the geometry tables (same layout as the front of the device array)
alignas(256) static unsigned char g_noalloc_host[kNoAllocScratchBytes];
static void* g_noalloc_dev[kNoAllocMaxDevices];
// serialises the host side of every call: the staging buffer and the device-address table
// are process-wide (locking allocates nothing)
static std::mutex g_noalloc_mu;

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

static long long fixed32(double v) { return llrint(v * 4294967296.0); }

}  // namespace pget

using namespace pget;

static pget_status forward_noalloc(const pget_geometry* gin, int32_t precision, const void* lam, const void* mu,
                                   void* y, void* stream);

extern "C" pget_status pget_forward_noalloc(const pget_geometry* gin, int32_t precision, const void* lam,
                                            const void* mu, void* y, void* stream) {
    // no C++ exception crosses the C boundary (a failed mutex would throw)
    try {
        return forward_noalloc(gin, precision, lam, mu, y, stream);
    } catch (...) {
        return PGET_EINTERNAL;
    }
}

static pget_status forward_noalloc(const pget_geometry* gin, int32_t precision, const void* lam, const void* mu,
                                   void* y, void* stream) {
    if (!gin || !lam || !mu || !y) return PGET_EINVAL;
    if (gin->depth_w || gin->depth_c) return PGET_EINVAL;  // depth tables need a context workspace
    if (precision != PGET_F64 && precision != PGET_F32 && precision != PGET_F32_KAHAN) return PGET_EINVAL;
    const bool f64 = precision == PGET_F64;
    const size_t elt = f64 ? 8 : 4;
    cudaStream_t st = (cudaStream_t)stream;

    // ---- geometry (same definitions as the context path, computed without the heap)
    const int n = gin->n, na = gin->n_angles, nd = gin->n_det, S = gin->n_sub, col = gin->collimator;
    if (n < 2 || n > 16384 || na < 1 || na > kMaxAngles || nd < 1 || S < 1 || S > kMaxSub || (col != 0 && col != 1)) return PGET_EINVAL;
    const int nbk = gin->n_banks == 0 ? (nd == 182 ? 2 : 1) : gin->n_banks;
    if ((nbk != 1 && nbk != 2) || nd % nbk) return PGET_EINVAL;
    const int nb = nd / nbk;
    if (nb > kMaxSlots) return PGET_EINVAL;  // at least one distinct ray per detector
    const double h = gin->step > 0 ? gin->step : 1.0;
    const double r = gin->fov_radius > 0 ? gin->fov_radius : n / std::sqrt(2.0);
    const double p = gin->det_pitch > 0 ? gin->det_pitch : 2.0 * r / nb;
    if (!std::isfinite(h) || !std::isfinite(r) || !std::isfinite(p)) return PGET_EINVAL;
    const double Td = std::ceil(2.0 * r / h);
    if (Td < 1 || Td > (1 << 20)) return PGET_EINVAL;
    const int T = (int)Td;
    const double c = 0.5 * (n - 1);
    const double sigma = col == 1 ? p / (2.0 * (S + 1)) : p / (2.0 * S);
    auto lattice = [&](int b, int d, int k) -> long long {
        long long a = 2LL * d - nb + 1 + b;
        return col == 1 ? a * (S + 1) + 2LL * (2 * k - S + 1) : a * S + (2LL * k - S + 1);
    };
    long long mmin[2] = {0, 0}, gstep[2] = {1, 1};
    int nslots[2] = {0, 0}, max_slots = 0;
    for (int b = 0; b < nbk; ++b) {
        long long mn = lattice(b, 0, 0), mx = mn;
        for (int d = 0; d < nb; ++d)
            for (int k = 0; k < S; ++k) {
                long long m = lattice(b, d, k);
                mn = m < mn ? m : mn;
                mx = m > mx ? m : mx;
            }
        long long gg = 0;
        for (int d = 0; d < nb; ++d)
            for (int k = 0; k < S; ++k) gg = std::gcd(gg, lattice(b, d, k) - mn);
        if (gg == 0) gg = 1;
        long long ns = (mx - mn) / gg + 1;
        if (ns > kMaxSlots) return PGET_EINVAL;
        mmin[b] = mn;
        gstep[b] = gg;
        nslots[b] = (int)ns;
        max_slots = (int)ns > max_slots ? (int)ns : max_slots;
    }
    const int V = na * nbk;
    const int P = ((n + 2 + 1) / 2) * 2;
    const size_t img_bytes = (size_t)(n + 2) * P * 2 * elt;
    size_t off = 0;
    const size_t o_err = off;
    off = align256(off + 16);
    const size_t o_views = off;
    off = align256(off + sizeof(ViewDev) * (size_t)V);
    const size_t o_clip = off;
    off = align256(off + 8 * (size_t)V * max_slots);
    const size_t o_det = off;
    off = align256(off + 4 * (size_t)nd * S);
    const size_t o_w = off;
    off = align256(off + elt * (size_t)S);
    const size_t tables_end = off;
    const size_t o_img0 = off;
    off = align256(off + img_bytes);
    const size_t o_img1 = off;
    off = align256(off + img_bytes);
    if (off > kNoAllocScratchBytes) return PGET_ENOMEM;

    // a captured table copy would read the shared staging buffer at replay time
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return PGET_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return PGET_EINVAL;

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    // ---- per-device address of the scratch array (looked up once per device)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return PGET_ECUDA;
    if (!g_noalloc_dev[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PGET_ECUDA;
        g_noalloc_dev[dev] = ptr;
    }
    unsigned char* D = (unsigned char*)g_noalloc_dev[dev];
    unsigned char* H = g_noalloc_host;

    // ---- tables into the host staging buffer
    memset(H, 0, tables_end);
    ViewDev* views = (ViewDev*)(H + o_views);
    int* clip = (int*)(H + o_clip);
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nbk; ++b) {
            const double psi = 2.0 * M_PI * a / na + b * M_PI;
            const double ct = std::cos(psi), stn = std::sin(psi);
            const double s0 = mmin[b] * sigma, t0 = -r + 0.5 * h, ds = gstep[b] * sigma;
            double px = -s0 * stn + t0 * ct + c, py = s0 * ct + t0 * stn + c;
            double Dx = h * ct, Dy = h * stn, Rx = -ds * stn, Ry = ds * ct;
            ViewDev v;
            memset(&v, 0, sizeof v);
            v.transposed = std::fabs(ct) > std::fabs(stn);
            if (v.transposed) {
                std::swap(px, py);
                std::swap(Dx, Dy);
                std::swap(Rx, Ry);
            }
            v.flipped = Dy < 0;
            if (v.flipped) {
                py = (n - 1) - py;
                Dy = -Dy;
                Ry = -Ry;
            }
            v.X00d = px;
            v.Y00d = py;
            v.dXsd = Dx;
            v.dYsd = Dy;
            v.dXrd = Rx;
            v.dYrd = Ry;
            v.X00 = fixed32(px);
            v.Y00 = fixed32(py);
            v.dXs = fixed32(Dx);
            v.dYs = fixed32(Dy);
            v.dXr = fixed32(Rx);
            v.dYr = fixed32(Ry);
            v.bank = b;
            v.angle = a;
            v.n_slots = nslots[b];
            const int vv = a * nbk + b;
            views[vv] = v;
            for (int i = 0; i < max_slots; ++i) {
                int* cc = &clip[((size_t)vv * max_slots + i) * 2];
                cc[0] = 0;
                cc[1] = -1;
                if (i >= v.n_slots) continue;
                const double X0 = v.X00d + i * v.dXrd, Y0 = v.Y00d + i * v.dYrd;
                double lo = 0.0, hi = T - 1.0;
                lo = std::max(lo, std::ceil((-1.0 - Y0) / v.dYsd) - 1.0);
                hi = std::min(hi, std::floor((n - Y0) / v.dYsd) + 1.0);
                if (std::fabs(v.dXsd) > 1e-9) {
                    double lo2 = (-1.0 - X0) / v.dXsd, hi2 = (n - X0) / v.dXsd;
                    if (lo2 > hi2) std::swap(lo2, hi2);
                    lo = std::max(lo, std::ceil(lo2) - 1.0);
                    hi = std::min(hi, std::floor(hi2) + 1.0);
                } else if (X0 < -1.0 - 1e-6 || X0 > n + 1e-6) {
                    hi = lo - 1.0;
                }
                if (hi >= lo) {
                    cc[0] = (int)lo;
                    cc[1] = (int)hi;
                }
            }
        }
    int* det = (int*)(H + o_det);
    double wsum = 0.0;
    double wk[kMaxSub];
    for (int k = 0; k < S; ++k) {
        const double m = k - 0.5 * (S - 1);
        const double u = col == 1 ? m * 2.0 * p / (S + 1) : m * p / S;
        wk[k] = col == 1 ? 1.0 - std::fabs(u) / p : 1.0;
        wsum += wk[k];
    }
    for (int k = 0; k < S; ++k) {
        wk[k] /= wsum;
        if (f64) ((double*)(H + o_w))[k] = wk[k];
        else ((float*)(H + o_w))[k] = (float)wk[k];
    }
    for (int dd = 0; dd < nd; ++dd) {
        const int b = dd / nb, d = dd % nb;
        for (int k = 0; k < S; ++k) det[dd * S + k] = (int)((lattice(b, d, k) - mmin[b]) / gstep[b]);
    }

    // ---- device work: tables, zeroed image borders, packing, the forward walk
    if (cudaMemcpyAsync(D, H, tables_end, cudaMemcpyHostToDevice, st) != cudaSuccess) return PGET_ECUDA;
    if (cudaMemsetAsync(D + o_img0, 0, off - o_img0, st) != cudaSuccess) return PGET_ECUDA;
    void* img0 = D + o_img0;
    void* img1 = D + o_img1;
    const double kappa = h * 1.4426950408889634;  // h log2(e): attenuation in powers of 2
    if (f64) pack<double, double>((const double*)lam, (const double*)mu, n, P, kappa, img0, img1, nullptr, st);
    else pack<float, float>((const float*)lam, (const float*)mu, n, P, kappa, img0, img1, nullptr, st);
    Geometry gplan;  // scalar fields only (its containers stay empty)
    gplan.n = n;
    gplan.max_slots = max_slots;
    gplan.h = h;
    const WalkPlan pl = plan_walk(gplan, P, kFwd, f64, 64 * 1024);
    WalkArgs a;
    memset(&a, 0, sizeof a);
    a.views = (const ViewDev*)(D + o_views);
    a.n = n;
    a.T = T;
    a.P = P;
    a.Yc = pl.Yc;
    a.nchunks = pl.nchunks;
    a.h = h;
    a.u_img[0] = img0;
    a.u_img[1] = img1;
    a.max_slots = max_slots;
    a.n_det = nd;
    a.n_banks = nbk;
    a.nb = nb;
    a.n_sub = S;
    a.det_slot = (const int*)(D + o_det);
    a.w = D + o_w;
    a.clip = (const int2*)(D + o_clip);
    a.y_out = y;
    a.err = (int*)(D + o_err);
    if (launch_walk(kFwd, precision, pl, a, V, st) != cudaSuccess) return PGET_ECUDA;
    // the kernel's error word (zeroed with the tables above): wait for the projection and
    // read it into a stack word (a copy to pageable memory returns once it has completed)
    int err = 0;
    if (cudaMemcpyAsync(&err, D + o_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PGET_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PGET_ECUDA;
    if (err & 4) return PGET_ETIMEOUT;  // a chunk copy did not arrive in time: y is void
    if (err) return PGET_ECUDA;
    return PGET_OK;
}
