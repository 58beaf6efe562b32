// pget_internal.cuh -- shared definitions of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pget.h"

namespace pget {

constexpr int kMaxSub = 64;
constexpr int kMaxSlots = 1024;   // rays per bank and view handled by one CTA (one per thread)
constexpr int kMaxAngles = 1 << 20;  // views = angles x banks stay far inside int and the launch grid
constexpr size_t kMaxTableSlots = size_t(1) << 26;  // views x rays per view of the host tables (512 MB of clips)
constexpr int kWalkThreads = 896; // block bound of the walk kernels for views up to this size

// ---------------------------------------------------------------- geometry
//
// Every sub-ray offset s_d + u_k of a bank lies on the lattice sigma * Z with
// sigma = p / (2 (S + 1)) (triangular) or p / (2 S) (box); coinciding sub-rays of
// neighbouring detectors are the same ray, so each bank has n_slots distinct rays
// ("slots") at s = (m_min + i * g) * sigma, i = 0..n_slots-1, and a detector reading is
// the weighted sum of the slots its sub-rays fall on.  A "view" is one (angle, bank):
// all its rays are parallel, travelling along theta toward the detector.
//
// Canonical frame of a view: pixel-index coordinates (X, Y) chosen so that the rays
// advance at least as fast in Y as in X and Y grows toward the detector:
//   transposed:  (X, Y) = (fy, fx) when |cos psi| > |sin psi|, else (fx, fy);
//   flipped:     Y <- (n - 1) - Y when the ray would move toward smaller Y.
// Kernels walk each ray from the detector side (largest j, largest Y) downward.

struct ViewDev {
    // sample (slot i, j) sits at P00 + i * R + j * D in the canonical frame
    long long X00, Y00, dXs, dYs, dXr, dYr;   // 32.32 fixed point (FP32 paths)
    double X00d, Y00d, dXsd, dYsd, dXrd, dYrd;  // double (FP64 path and ray clipping)
    int transposed, flipped, bank, angle;
    int n_slots;
    int pad;
};

struct Geometry {
    int n = 0, n_angles = 0, n_det = 0, n_banks = 0, nb = 0, n_sub = 0, collimator = 0;
    double h = 1, r = 0, p = 0, c = 0;
    int T = 0;
    double sigma = 0;
    int m_min[2] = {0, 0}, g[2] = {1, 1}, n_slots[2] = {0, 0};
    int max_slots = 0;
    std::vector<double> w;            // [S] sub-ray weights
    std::vector<int> det_slot;        // [n_det][S] slot of each sub-ray (in its bank)
    // per (bank, slot): sub-rays landing on it, CSR over (bank * max_slots + slot)
    std::vector<int> src_off;         // [n_banks * max_slots + 1]
    std::vector<int> src_det;         // detector index within [0, n_det)
    std::vector<double> src_w;        // its weight
    std::vector<ViewDev> views;       // [n_angles * n_banks], view v = a * n_banks + b
    // per (view, slot): conservative sample range [jlo, jhi] whose base pixel can lie in
    // [-1, n-1]^2 (the kernels test every sample exactly); empty rays have jhi < jlo
    std::vector<int> clip;            // [n_views * max_slots * 2]
    int views_transposed = 0;
    // depth factors of Eq. (5), [T] each, empty without tables: sample j contributes
    // h w_j lambda_j exp(-c_j E_j)
    std::vector<double> depth_w, depth_c;
    bool depth = false;
    std::string key;                  // identifies the geometry for workspace caching
};

// Resolve defaults, validate, build the slot tables and the per-view frames.
// Returns PGET_OK or PGET_EINVAL with *msg set.
pget_status build_geometry(const pget_geometry& in, Geometry* out, std::string* msg);

}  // namespace pget
