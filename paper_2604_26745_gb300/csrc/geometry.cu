// geometry.cu -- host-side resolution of the measurement geometry into per-view frames
// and the sub-ray -> slot tables used by the kernels.
//
// The geometry is the one of Sec. 2 / Sec. 2.1 of the paper (two opposed detector banks
// with a half-pitch offset over a full rotation, collimated detectors, rays ending at a
// detector at s theta_perp + r theta), sampled as the discrete model of Eq. (5).
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>

#include "pget_internal.cuh"

namespace pget {

static long long to_fixed(double v) { return llrint(v * 4294967296.0); }

pget_status build_geometry(const pget_geometry& in, Geometry* G, std::string* msg) {
    Geometry g;
    g.n = in.n;
    g.n_angles = in.n_angles;
    g.n_det = in.n_det;
    g.n_sub = in.n_sub;
    g.collimator = in.collimator;
    if (g.n < 2 || g.n > 16384) return *msg = "n must be in [2, 16384]", PGET_EINVAL;
    if (g.n_angles < 1 || g.n_angles > kMaxAngles) return *msg = "n_angles must be in [1, 1048576]", PGET_EINVAL;
    if (g.n_det < 1) return *msg = "n_det must be >= 1", PGET_EINVAL;
    if (g.n_sub < 1 || g.n_sub > kMaxSub) return *msg = "n_sub must be in [1, 64]", PGET_EINVAL;
    if (g.collimator != 0 && g.collimator != 1) return *msg = "collimator must be 0 or 1", PGET_EINVAL;
    g.n_banks = in.n_banks == 0 ? (g.n_det == 182 ? 2 : 1) : in.n_banks;
    if (g.n_banks != 1 && g.n_banks != 2) return *msg = "n_banks must be 1 or 2", PGET_EINVAL;
    if (g.n_det % g.n_banks) return *msg = "n_det must be a multiple of n_banks", PGET_EINVAL;
    g.nb = g.n_det / g.n_banks;
    // every detector of a bank adds at least one distinct ray: refuse before any table
    // is sized by the detector count
    if (g.nb > kMaxSlots) return *msg = "more than 1024 detectors per bank", PGET_EINVAL;
    g.h = in.step > 0 ? in.step : 1.0;
    g.r = in.fov_radius > 0 ? in.fov_radius : g.n / std::sqrt(2.0);
    g.p = in.det_pitch > 0 ? in.det_pitch : 2.0 * g.r / g.nb;
    if (!std::isfinite(g.h) || !std::isfinite(g.r) || !std::isfinite(g.p))
        return *msg = "non-finite step, fov_radius or det_pitch", PGET_EINVAL;
    double Td = std::ceil(2.0 * g.r / g.h);
    if (Td < 1 || Td > 1 << 20) return *msg = "samples per ray out of range", PGET_EINVAL;
    g.T = (int)Td;
    g.c = 0.5 * (g.n - 1);
    if (in.depth_w || in.depth_c) {
        g.depth = true;
        g.depth_w.assign(g.T, 1.0);
        g.depth_c.assign(g.T, 1.0);
        for (int j = 0; j < g.T; ++j) {
            if (in.depth_w) g.depth_w[j] = in.depth_w[j];
            if (in.depth_c) g.depth_c[j] = in.depth_c[j];
            if (!(std::isfinite(g.depth_w[j]) && g.depth_w[j] >= 0.0 && std::isfinite(g.depth_c[j]) &&
                  g.depth_c[j] >= 0.0))
                return *msg = "depth tables must be finite and >= 0", PGET_EINVAL;
        }
    }
    const int S = g.n_sub;

    // sub-ray weights
    g.w.resize(S);
    double tot = 0.0;
    for (int k = 0; k < S; ++k) {
        double m = k - 0.5 * (S - 1);
        double u = g.collimator == 1 ? m * 2.0 * g.p / (S + 1) : m * g.p / S;
        g.w[k] = g.collimator == 1 ? 1.0 - std::fabs(u) / g.p : 1.0;
        tot += g.w[k];
    }
    for (int k = 0; k < S; ++k) g.w[k] /= tot;

    // integer lattice index of every sub-ray: s = m * sigma
    g.sigma = g.collimator == 1 ? g.p / (2.0 * (S + 1)) : g.p / (2.0 * S);
    std::vector<long long> m_of((size_t)g.n_det * S);
    for (int b = 0; b < g.n_banks; ++b) {
        long long mn = 0, mx = 0;
        bool first = true;
        for (int d = 0; d < g.nb; ++d)
            for (int k = 0; k < S; ++k) {
                long long a = 2LL * d - g.nb + 1 + b;
                long long m = g.collimator == 1 ? a * (S + 1) + 2LL * (2 * k - S + 1)
                                                 : a * S + (2LL * k - S + 1);
                m_of[((size_t)b * g.nb + d) * S + k] = m;
                if (first || m < mn) mn = m;
                if (first || m > mx) mx = m;
                first = false;
            }
        long long gg = 0;
        for (int d = 0; d < g.nb; ++d)
            for (int k = 0; k < S; ++k) gg = std::gcd(gg, m_of[((size_t)b * g.nb + d) * S + k] - mn);
        if (gg == 0) gg = 1;
        long long ns = (mx - mn) / gg + 1;
        if (ns > kMaxSlots) {
            char buf[160];
            snprintf(buf, sizeof buf, "geometry needs %lld distinct rays per view (limit %d)", ns, kMaxSlots);
            return *msg = buf, PGET_EINVAL;
        }
        g.m_min[b] = (int)mn;
        g.g[b] = (int)gg;
        g.n_slots[b] = (int)ns;
        g.max_slots = std::max(g.max_slots, (int)ns);
    }
    g.det_slot.resize((size_t)g.n_det * S);
    std::vector<std::vector<std::pair<int, double>>> src((size_t)g.n_banks * g.max_slots);
    for (int dd = 0; dd < g.n_det; ++dd) {
        int b = dd / g.nb;
        for (int k = 0; k < S; ++k) {
            long long m = m_of[(size_t)dd * S + k];
            int slot = (int)((m - g.m_min[b]) / g.g[b]);
            g.det_slot[(size_t)dd * S + k] = slot;
            src[(size_t)b * g.max_slots + slot].push_back({dd, g.w[k]});
        }
    }
    g.src_off.assign(src.size() + 1, 0);
    for (size_t q = 0; q < src.size(); ++q) {
        g.src_off[q + 1] = g.src_off[q] + (int)src[q].size();
        for (auto& e : src[q]) {
            g.src_det.push_back(e.first);
            g.src_w.push_back(e.second);
        }
    }

    // per-view canonical frames; the view and clip tables grow with views x slots
    if ((size_t)g.n_angles * g.n_banks * g.max_slots > kMaxTableSlots)
        return *msg = "geometry tables too large (views x rays per view above 2^26)", PGET_ENOMEM;
    g.views.resize((size_t)g.n_angles * g.n_banks);
    g.views_transposed = 0;
    for (int a = 0; a < g.n_angles; ++a)
        for (int b = 0; b < g.n_banks; ++b) {
            double psi = 2.0 * M_PI * a / g.n_angles + b * M_PI;
            double ct = std::cos(psi), st = std::sin(psi);
            double s0 = g.m_min[b] * g.sigma, t0 = -g.r + 0.5 * g.h, ds = g.g[b] * g.sigma;
            // pixel-index coordinates of sample (slot 0, j = 0) and the steps
            double px = -s0 * st + t0 * ct + g.c, py = s0 * ct + t0 * st + g.c;
            double Dx = g.h * ct, Dy = g.h * st;
            double Rx = -ds * st, Ry = ds * ct;
            ViewDev v{};
            v.transposed = std::fabs(ct) > std::fabs(st);
            if (v.transposed) {
                std::swap(px, py);
                std::swap(Dx, Dy);
                std::swap(Rx, Ry);
            }
            v.flipped = Dy < 0;
            if (v.flipped) {
                py = (g.n - 1) - py;
                Dy = -Dy;
                Ry = -Ry;
            }
            v.X00d = px;
            v.Y00d = py;
            v.dXsd = Dx;
            v.dYsd = Dy;
            v.dXrd = Rx;
            v.dYrd = Ry;
            v.X00 = to_fixed(px);
            v.Y00 = to_fixed(py);
            v.dXs = to_fixed(Dx);
            v.dYs = to_fixed(Dy);
            v.dXr = to_fixed(Rx);
            v.dYr = to_fixed(Ry);
            v.bank = b;
            v.angle = a;
            v.n_slots = g.n_slots[b];
            g.views[(size_t)a * g.n_banks + b] = v;
            g.views_transposed += v.transposed;
        }
    // conservative per-ray sample ranges (host double arithmetic, once per geometry)
    g.clip.assign((size_t)g.views.size() * g.max_slots * 2, 0);
    for (size_t vv = 0; vv < g.views.size(); ++vv) {
        const ViewDev& v = g.views[vv];
        for (int i = 0; i < g.max_slots; ++i) {
            int* c = &g.clip[(vv * g.max_slots + i) * 2];
            c[0] = 0;
            c[1] = -1;
            if (i >= v.n_slots) continue;
            double X0 = v.X00d + i * v.dXrd, Y0 = v.Y00d + i * v.dYrd;
            double lo = 0.0, hi = g.T - 1.0;
            lo = std::max(lo, std::ceil((-1.0 - Y0) / v.dYsd) - 1.0);
            hi = std::min(hi, std::floor((g.n - Y0) / v.dYsd) + 1.0);
            if (std::fabs(v.dXsd) > 1e-9) {
                double a = (-1.0 - X0) / v.dXsd, b = (g.n - X0) / v.dXsd;
                if (a > b) std::swap(a, b);
                lo = std::max(lo, std::ceil(a) - 1.0);
                hi = std::min(hi, std::floor(b) + 1.0);
            } else if (X0 < -1.0 - 1e-6 || X0 > g.n + 1e-6) {
                hi = lo - 1.0;
            }
            if (hi >= lo) {
                c[0] = (int)lo;
                c[1] = (int)hi;
            }
        }
    }
    char key[320];
    int kl = snprintf(key, sizeof key, "%d/%d/%d/%d/%d/%d/%.17g/%.17g/%.17g", g.n, g.n_angles, g.n_det,
                      g.n_banks, g.n_sub, g.collimator, g.h, g.r, g.p);
    if (g.depth) {  // the tables' contents are part of the geometry (FNV-1a over their bytes)
        unsigned long long hsh = 1469598103934665603ull;
        for (const std::vector<double>* tab : {&g.depth_w, &g.depth_c}) {
            const unsigned char* b = (const unsigned char*)tab->data();
            for (size_t i = 0; i < tab->size() * sizeof(double); ++i) hsh = (hsh ^ b[i]) * 1099511628211ull;
        }
        snprintf(key + kl, sizeof key - kl, "/depth:%016llx", hsh);
    }
    g.key = key;
    *G = std::move(g);
    return PGET_OK;
}

}  // namespace pget
