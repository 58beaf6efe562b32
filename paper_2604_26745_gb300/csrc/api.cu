// api.cu -- the C ABI of libpget.so: context, workspace, and the drivers of the
// forward / JVP / VJP operators, the CG solve of Eq. (9) and the LM iteration (Sec. 2.2).
#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"
#include "pget_internal.cuh"
#include "vec.cuh"

using namespace pget;

static thread_local std::string g_last_error;

static bool known_precision(int p) {
    return p == PGET_F64 || p == PGET_F32 || p == PGET_F32_KAHAN || p == PGET_MIXED;
}
// the precision of the ray kernels (walks) for a solver precision
static int walk_precision(int p) { return p == PGET_MIXED ? PGET_F32_KAHAN : p; }
// solver vectors (iterate, data, CG and LM vectors) in double
static bool vectors_f64(int p) { return p == PGET_F64 || p == PGET_MIXED; }

static pget_status fail(pget_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    try {
        g_last_error = buf;
    } catch (...) {  // out of host memory: the status still reports the failure
    }
    return s;
}

// Every pget_status entry point runs its body through guarded(): a host-side exception (a
// failed host allocation, a failed mutex) becomes a status instead of crossing the C
// boundary, where it would end the caller's process.
template <typename F>
static pget_status guarded(F&& body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return fail(PGET_ENOMEM, "host memory allocation failed");
    } catch (const std::exception& e) {
        return fail(PGET_EINTERNAL, "internal error: %s", e.what());
    } catch (...) {
        return fail(PGET_EINTERNAL, "internal error");
    }
}

// Host-side NVTX range around a public call, for profilers that show or filter by them
// (Nsight Systems timelines, ncu's --nvtx-include); without a tool attached it does nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define PGET_RANGE(name) NvtxRange nvtx_range_(name)

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(PGET_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

namespace pget {

// -------------------------------------------------------------------- profiling
// CUDA events around the hot kernels, recorded on the stream the kernels run on;
// elapsed times are collected once the stream has been synchronised.
enum ProfKind { kPFwd = 0, kPJvp = 1, kPVjp = 2, kPRed = 3, kPKinds = 4 };
static const char* kProfNames[kPKinds] = {"walk_forward", "walk_jvp", "walk_vjp", "reduce_views"};

struct Profiler {
    bool on = false;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double total_ms[kPKinds] = {0, 0, 0, 0};
    long long count[kPKinds] = {0, 0, 0, 0};
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    bool capturing = false;        // records become event nodes of a CUDA graph
    std::vector<Rec> captured;
    void begin(int kind, cudaStream_t st) {
        if (!on) return;
        Rec r{kind, get(), get()};
        if (capturing) {
            cudaEventRecordWithFlags(r.a, st, cudaEventRecordExternal);
            captured.push_back(r);
        } else {
            cudaEventRecord(r.a, st);
            pending.push_back(r);
        }
    }
    void end(cudaStream_t st) {
        if (!on) return;
        if (capturing) {
            if (!captured.empty()) cudaEventRecordWithFlags(captured.back().b, st, cudaEventRecordExternal);
        } else if (!pending.empty()) {
            cudaEventRecord(pending.back().b, st);
        }
    }
    // after a replay of a graph captured with profiling on (stream synchronised)
    void collect_graph(const std::vector<Rec>& recs) {
        for (auto& r : recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                total_ms[r.kind] += ms;
                count[r.kind] += 1;
            }
        }
    }
    void collect() {
        for (auto& r : pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                total_ms[r.kind] += ms;
                count[r.kind] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    void reset() {
        collect();
        for (int k = 0; k < kPKinds; ++k) {
            total_ms[k] = 0;
            count[k] = 0;
        }
    }
    ~Profiler() {
        for (auto& r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// --------------------------------------------------------------------- workspace
struct Workspace {
    Profiler* prof = nullptr;
    Geometry g;
    int prec = 0;
    bool f64 = false;     // solver vectors in double
    size_t elt = 4;       // bytes of a solver vector element
    int wprec = 0;        // precision of the ray kernels (walks)
    bool wf64 = false;    // walk images, ray totals and partial images in double
    size_t welt = 4;      // bytes of a walk element
    void* sino_w = nullptr;  // PGET_MIXED: a sinogram in the walks' type
    // PGET_MIXED: the objective's forward model in double: its plan, packed layouts, ray
    // totals (narrowed to the float ones the adjoint reads) and weight tables
    bool obj64 = false;
    WalkPlan pf64;
    void* pk64[2] = {nullptr, nullptr};
    void *U64 = nullptr, *d_w64 = nullptr, *d_depth64 = nullptr;
    int P = 0, groups = 1, n_views = 0;
    size_t nn = 0, M = 0, nslots = 0, img_elems = 0;
    WalkPlan pf, pj, pv;
    ViewDev* d_views = nullptr;
    int* d_det_slot = nullptr;
    void* d_w = nullptr;        // sub-ray weights in the element type of the path
    int* d_src_off = nullptr;
    int* d_src_det = nullptr;
    void* d_src_w = nullptr;    // per-slot sub-ray weights in the element type of the path
    int2* d_clip = nullptr;
    int2* d_win = nullptr;       // adjoint ray windows [view][chunk]
    // test aids of the failure path (0 in normal use): extra expected bytes on the first
    // chunk copy of every walk, and the chunk-copy wait limit
    int tx_extra = 0;
    long long wait_ns = 0;
    // adjoint view groups: CTA g sums views group_view[group_off[g] .. group_off[g+1]),
    // all of one canonical orientation, into partial image g
    int n_groups = 0, n_groups0 = 0;  // CTA groups in all / in the normal frame (listed first)
    void* d_depth = nullptr;  // [T] (w_j, c_j) depth factors of Eq. (5), element type; null without
    int* d_group_off = nullptr;
    int* d_group_view = nullptr;
    // launch orders: CTA b of a forward or JVP walk takes view d_view_order[b], CTA b of an
    // adjoint walk group d_group_order[b], longest rays first (see walk_orders)
    int* d_view_order = nullptr;
    int* d_group_order = nullptr;
    void* pk_u[2] = {nullptr, nullptr};
    void* pk_ut[2] = {nullptr, nullptr};
    void* pk_p[2] = {nullptr, nullptr};
    void *u = nullptr, *ut = nullptr, *x = nullptr, *res = nullptr, *p = nullptr, *q = nullptr,
         *s = nullptr, *gr = nullptr, *Wl = nullptr, *Wm = nullptr;
    void *yb = nullptr, *r = nullptr, *rt = nullptr, *Jp = nullptr;
    void *U = nullptr, *Ut = nullptr;
    void *gpart = nullptr, *part2 = nullptr;
    double* dpart[4] = {nullptr, nullptr, nullptr, nullptr};
    LmState* lm = nullptr;
    int* err = nullptr;
    std::vector<void*> allocs;
    size_t bytes = 0;
    // CUDA graph of the LM body (everything between the input copies and the result copy)
    cudaStream_t cap_stream = nullptr;
    LmState* host_lm = nullptr;      // pinned copy of the device LM state after a solve
    int* host_err = nullptr;         // pinned copy of the device error flags
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // solve timing (stream events)
    std::string graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<Profiler::Rec> graph_events;
    long long graph_launches = 0;
    bool graph_used = false;

    ~Workspace() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        for (auto& r : graph_events) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (host_lm) cudaFreeHost(host_lm);
        if (host_err) cudaFreeHost(host_err);
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
        for (void* a : allocs) cudaFree(a);
    }
    template <typename X>
    cudaError_t alloc(X** ptr, size_t bytes_) {
        void* a = nullptr;
        size_t b = bytes_ ? bytes_ : 16;
        cudaError_t e = cudaMalloc(&a, b);
        if (e != cudaSuccess) return e;
        allocs.push_back(a);
        bytes += b;
        *ptr = (X*)a;
        return cudaMemset(a, 0, b);
    }
};

// bytes a workspace for this geometry and precision will take
static size_t workspace_bytes(const Geometry& g, int prec, int groups) {
    size_t elt = vectors_f64(prec) ? 8 : 4, welt = walk_precision(prec) == PGET_F64 ? 8 : 4;
    size_t nn = (size_t)g.n * g.n, M = (size_t)g.n_angles * g.n_det;
    size_t V = (size_t)g.n_angles * g.n_banks;
    size_t P = (size_t)((g.n + 2 + 1) / 2) * 2;
    size_t img = (size_t)(g.n + 2) * P * 2 * welt;
    size_t b = 0;
    b += 6 * img;                       // three packed pairs, two layouts each
    b += 8 * 2 * nn * elt + 2 * nn * elt;  // vectors + weights
    b += 4 * M * elt + (elt != welt ? M * welt : 0);  // sinograms
    b += 2 * V * g.max_slots * welt;    // slot totals
    b += V * 2 * nn * welt;             // per-view partial gradients
    b += (size_t)groups * 2 * nn * welt;
    b += 4 * kRedBlocks * 8 + sizeof(LmState) + 64;
    b += V * sizeof(ViewDev) + V * 4 + (size_t)g.n_det * g.n_sub * 4 + g.n_sub * 8;
    b += 4 * (V + 1) * 4;               // view groups and the two launch orders
    b += g.src_off.size() * 4 + g.src_det.size() * 12 + g.clip.size() * 4;
    b += V * (size_t)(g.n + 1) * 8;     // adjoint ray windows (at most n + 1 chunks per view)
    if (g.depth) b += 2 * (size_t)g.T * welt;  // depth factors
    if (prec == PGET_MIXED)  // the objective's double forward: layouts, ray totals, tables
        b += (size_t)(g.n + 2) * P * 2 * 16 + 8 * V * (size_t)g.max_slots + 16 * (size_t)g.T + 8 * g.n_sub;
    return b;
}

}  // namespace pget

namespace pget {
// One in-flight reconstruction of the serving path: its own workspace (kept for reuse
// while the slot is free), stream, captured LM graph and completion event.
struct Slot {
    enum State { kFree = 0, kRunning = 1, kDone = 2 };
    int state = kFree;
    uint64_t ticket = 0;
    std::unique_ptr<Workspace> ws;
    std::string ws_key;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    pget_status launch_status = PGET_OK;
    ~Slot() {
        if (stream) cudaStreamSynchronize(stream);
        ws.reset();
        if (done) cudaEventDestroy(done);
        if (stream) cudaStreamDestroy(stream);
    }
};
}  // namespace pget

namespace pget {
// Buffers of the batched operator calls for one workspace: the packed layouts (iterate
// and direction), ray totals, a scratch sinogram and the adjoint partial images of `cap`
// items at once.
struct BatchBufs {
    std::string key;
    int cap = 0;
    long long s_img = 0, s_slot = 0, s_sino = 0, s_part = 0;  // bytes per item
    void *pk_u[2] = {nullptr, nullptr}, *pk_p[2] = {nullptr, nullptr};
    void *U = nullptr, *sino = nullptr, *gpart = nullptr;
    std::vector<void*> allocs;
    ~BatchBufs() {
        for (void* a : allocs) cudaFree(a);
    }
};
constexpr size_t kBatchPartBytes = size_t(4) << 30;  // adjoint partial images of one chunk of items
}  // namespace pget

struct pget_ctx {
    Profiler prof;
    std::unique_ptr<pget::BatchBufs> batch;
    std::vector<std::unique_ptr<pget::Slot>> slots;
    // idle serving workspaces (with their captured graphs), reused by geometry key so that
    // a stream of mixed sizes does not allocate and free device memory per request
    struct Idle {
        std::string key;
        std::unique_ptr<pget::Workspace> ws;
        uint64_t last_use = 0;
    };
    std::vector<Idle> pool;
    uint64_t use_clock = 0;
    uint64_t next_ticket = 1;
    int device = 0;
    size_t budget = 0;
    std::mutex mu;
    std::unique_ptr<Workspace> ws;
    std::string ws_key;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Resolve and validate a geometry; the key identifies (geometry, precision).
pget_status resolve(const pget_geometry* gin, int prec, Geometry* g, std::string* key, int* groups,
                    size_t* need) {
    if (!gin) return fail(PGET_EINVAL, "null geometry");
    if (!known_precision(prec)) return fail(PGET_EINVAL, "unknown precision %d", prec);
    std::string msg;
    pget_status s = build_geometry(*gin, g, &msg);
    if (s != PGET_OK) return fail(s, "%s", msg.c_str());
    *key = g->key + "#" + std::to_string(prec);
    const int V = g->n_angles * g->n_banks;
    const int tiles = ((g->n + 31) / 32) * ((g->n + 31) / 32);
    *groups = std::max(1, std::min(V, (2 * kRedBlocks + tiles - 1) / tiles));
    *need = workspace_bytes(*g, prec, *groups);
    return PGET_OK;
}

// Launch orders of the walks.  A walk CTA's time grows with the length of its view's
// rays (their samples per image row go as 1/cos of the ray's angle to the canonical
// axis: up to sqrt(2) times more at 45 degrees), and a launch of more CTAs than fit at
// once ends with a partial wave.  Launching the longest views first leaves the shortest
// for that wave (longest-processing-time-first list scheduling); ties keep the view
// order.  Every view or group still writes its own output, so results do not change.
void walk_orders(const Geometry& G, const std::vector<int>& goff, const std::vector<int>& gview,
                 std::vector<int>* vorder, std::vector<int>* gorder) {
    const int V = (int)G.views.size(), ms = G.max_slots;
    std::vector<long long> len(V, 0);  // samples of the view's longest ray
    for (int v = 0; v < V; ++v)
        for (int i = 0; i < G.views[v].n_slots; ++i) {
            const long long lo = G.clip[((size_t)v * ms + i) * 2], hi = G.clip[((size_t)v * ms + i) * 2 + 1];
            len[v] = std::max(len[v], hi - lo + 1);
        }
    const int NG = (int)goff.size() - 1;
    std::vector<long long> glen(NG, 0);
    for (int g = 0; g < NG; ++g)
        for (int k = goff[g]; k < goff[g + 1]; ++k) glen[g] += len[gview[k]];
    auto order = [](const std::vector<long long>& c, std::vector<int>* o) {
        o->resize(c.size());
        for (size_t i = 0; i < c.size(); ++i) (*o)[i] = (int)i;
        std::stable_sort(o->begin(), o->end(), [&](int a, int b) { return c[a] > c[b]; });
    };
    order(len, vorder);
    order(glen, gorder);
}

size_t serving_bytes(const pget_ctx* ctx);
bool evict_idle(pget_ctx* ctx);

// Shared memory per walk CTA: three CTAs of up to 1024 threads share an SM's 227 KB (a
// build with -DPGET_TUNING reads PGET_SMEM_KB_{FWD,JVP,VJP} to sweep the budgets).
static size_t walk_budget(const char* env, size_t kb) {
#ifdef PGET_TUNING
    const char* v = getenv(env);
    if (v && atoi(v) > 0) kb = (size_t)atoi(v);
#else
    (void)env;
#endif
    return kb * 1024;
}

// The launch plans of the forward, JVP and adjoint walks (host only).
static void walk_plans(const Geometry& G, int P, bool wf64, WalkPlan* pf, WalkPlan* pj, WalkPlan* pv) {
    *pf = plan_walk(G, P, kFwd, wf64, walk_budget("PGET_SMEM_KB_FWD", 64));
    *pj = plan_walk(G, P, kJvp, wf64, walk_budget("PGET_SMEM_KB_JVP", 72));
    std::vector<int2> rows;
    ray_rows(G, wf64, &rows);
    *pv = plan_walk(G, P, kVjp, wf64, walk_budget("PGET_SMEM_KB_VJP", 72), &rows);
}

// Allocate and initialise a workspace for a resolved geometry (no budget check).
pget_status make_workspace(pget_ctx* ctx, Geometry&& g, int prec, int groups, std::unique_ptr<Workspace>* out) {
    const int V = g.n_angles * g.n_banks;
    auto w = std::make_unique<Workspace>();
    w->g = std::move(g);
    Geometry& G = w->g;
    w->prec = prec;
    w->f64 = vectors_f64(prec);
    w->elt = w->f64 ? 8 : 4;
    w->wprec = walk_precision(prec);
    w->wf64 = w->wprec == PGET_F64;
    w->welt = w->wf64 ? 8 : 4;
    w->obj64 = prec == PGET_MIXED;
    w->P = ((G.n + 2 + 1) / 2) * 2;
    w->groups = groups;
    w->n_views = V;
    w->nn = (size_t)G.n * G.n;
    w->M = (size_t)G.n_angles * G.n_det;
    w->nslots = (size_t)V * G.max_slots;
    w->img_elems = (size_t)(G.n + 2) * w->P;
    walk_plans(G, w->P, w->wf64, &w->pf, &w->pj, &w->pv);
    if (w->obj64) w->pf64 = plan_walk(G, w->P, kFwd, true, walk_budget("PGET_SMEM_KB_FWD", 64));
    // views per adjoint CTA: one (the hardware scheduler balances single-view CTAs across
    // SMs best); a build with -DPGET_TUNING reads PGET_VJP_VIEWS_PER_CTA > 1 to group views
    // of one orientation, which shrinks the partial images but assigns work statically (0
    // sizes groups so that every CTA is resident at once)
    int K = 1;
#ifdef PGET_TUNING
    if (const char* kv = getenv("PGET_VJP_VIEWS_PER_CTA")) {
        K = atoi(kv);
        if (K <= 0) {
            int sms = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
            const int slots = std::max(1, sms * walk_occupancy(kVjp, prec, w->pv));
            K = std::max(1, (V + slots - 1) / slots);
        }
    }
#endif
    std::vector<int> goff{0}, gview, gtrans;
    for (int cls = 0; cls < 2; ++cls) {
        std::vector<int> vs;
        for (int v = 0; v < V; ++v)
            if (G.views[v].transposed == cls) vs.push_back(v);
        for (size_t i = 0; i < vs.size(); i += K) {
            for (size_t k = i; k < std::min(vs.size(), i + (size_t)K); ++k) gview.push_back(vs[k]);
            goff.push_back((int)gview.size());
            gtrans.push_back(cls);
        }
    }
    w->n_groups = (int)gtrans.size();
    w->n_groups0 = (int)std::count(gtrans.begin(), gtrans.end(), 0);  // normal-frame groups come first
    std::vector<int> vorder, gorder;
    walk_orders(G, goff, gview, &vorder, &gorder);
    const size_t e = w->elt, we = w->welt;  // solver and walk element bytes
    CK(w->alloc(&w->d_views, sizeof(ViewDev) * V));
    CK(cudaMemcpy(w->d_views, G.views.data(), sizeof(ViewDev) * V, cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_det_slot, sizeof(int) * G.det_slot.size()));
    CK(cudaMemcpy(w->d_det_slot, G.det_slot.data(), sizeof(int) * G.det_slot.size(), cudaMemcpyHostToDevice));
    auto upload_t = [&](void** dst, const std::vector<double>& src) -> cudaError_t {
        cudaError_t er = w->alloc(dst, we * src.size());
        if (er != cudaSuccess) return er;
        if (w->wf64) return cudaMemcpy(*dst, src.data(), 8 * src.size(), cudaMemcpyHostToDevice);
        std::vector<float> f(src.begin(), src.end());
        return cudaMemcpy(*dst, f.data(), 4 * f.size(), cudaMemcpyHostToDevice);
    };
    CK(upload_t(&w->d_w, G.w));
    if (w->obj64) {  // the double tables of the objective's forward model
        CK(w->alloc(&w->d_w64, 8 * G.w.size()));
        CK(cudaMemcpy(w->d_w64, G.w.data(), 8 * G.w.size(), cudaMemcpyHostToDevice));
        if (G.depth) {
            std::vector<double> dt(2 * (size_t)G.T);
            for (int j = 0; j < G.T; ++j) {
                dt[2 * j] = G.depth_w[j];
                dt[2 * j + 1] = G.depth_c[j];
            }
            CK(w->alloc(&w->d_depth64, 8 * dt.size()));
            CK(cudaMemcpy(w->d_depth64, dt.data(), 8 * dt.size(), cudaMemcpyHostToDevice));
        }
        for (int l = 0; l < 2; ++l) CK(w->alloc(&w->pk64[l], 16 * w->img_elems));
        CK(w->alloc(&w->U64, 8 * w->nslots));
    }
    if (G.depth) {  // interleaved (w_j, c_j) pairs
        std::vector<double> dt(2 * (size_t)G.T);
        for (int j = 0; j < G.T; ++j) {
            dt[2 * j] = G.depth_w[j];
            dt[2 * j + 1] = G.depth_c[j];
        }
        CK(upload_t(&w->d_depth, dt));
    }
    CK(w->alloc(&w->d_clip, sizeof(int) * G.clip.size()));
    CK(cudaMemcpy(w->d_clip, G.clip.data(), sizeof(int) * G.clip.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_win, sizeof(int2) * w->pv.win.size()));
    CK(cudaMemcpy(w->d_win, w->pv.win.data(), sizeof(int2) * w->pv.win.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_src_off, sizeof(int) * G.src_off.size()));
    CK(cudaMemcpy(w->d_src_off, G.src_off.data(), sizeof(int) * G.src_off.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_src_det, sizeof(int) * G.src_det.size()));
    CK(cudaMemcpy(w->d_src_det, G.src_det.data(), sizeof(int) * G.src_det.size(), cudaMemcpyHostToDevice));
    CK(upload_t(&w->d_src_w, G.src_w));
    for (int l = 0; l < 2; ++l) {
        CK(w->alloc(&w->pk_u[l], 2 * we * w->img_elems));
        CK(w->alloc(&w->pk_ut[l], 2 * we * w->img_elems));
        CK(w->alloc(&w->pk_p[l], 2 * we * w->img_elems));
    }
    void** vecs[] = {&w->u, &w->ut, &w->x, &w->res, &w->p, &w->q, &w->s, &w->gr};
    for (void** vp : vecs) CK(w->alloc(vp, e * 2 * w->nn));
    CK(w->alloc(&w->Wl, e * w->nn));
    CK(w->alloc(&w->Wm, e * w->nn));
    CK(w->alloc(&w->yb, e * w->M));
    CK(w->alloc(&w->r, e * w->M));
    CK(w->alloc(&w->rt, e * w->M));
    CK(w->alloc(&w->Jp, e * w->M));
    if (we != e) CK(w->alloc(&w->sino_w, we * w->M));
    CK(w->alloc(&w->U, we * w->nslots));
    CK(w->alloc(&w->Ut, we * w->nslots));
    CK(w->alloc(&w->gpart, we * (size_t)w->n_groups * 2 * w->nn));
    CK(w->alloc(&w->d_group_off, sizeof(int) * goff.size()));
    CK(cudaMemcpy(w->d_group_off, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_group_view, sizeof(int) * gview.size()));
    CK(cudaMemcpy(w->d_group_view, gview.data(), sizeof(int) * gview.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_view_order, sizeof(int) * vorder.size()));
    CK(cudaMemcpy(w->d_view_order, vorder.data(), sizeof(int) * vorder.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->d_group_order, sizeof(int) * gorder.size()));
    CK(cudaMemcpy(w->d_group_order, gorder.data(), sizeof(int) * gorder.size(), cudaMemcpyHostToDevice));
    CK(w->alloc(&w->part2, we * (size_t)groups * 2 * w->nn));
    for (int k = 0; k < 4; ++k) CK(w->alloc(&w->dpart[k], sizeof(double) * kRedBlocks));
    CK(w->alloc(&w->lm, sizeof(LmState)));
    CK(w->alloc(&w->err, sizeof(int) * 4));
    CK(cudaMallocHost(&w->host_lm, sizeof(LmState)));
    CK(cudaMallocHost(&w->host_err, sizeof(int) * 4));
    CK(cudaEventCreate(&w->t0));
    CK(cudaEventCreate(&w->t1));
    if (const char* v = getenv("PGET_TEST_TX_EXTRA")) w->tx_extra = std::max(0, atoi(v)) / 16 * 16;
    if (const char* v = getenv("PGET_TEST_WAIT_NS")) w->wait_ns = std::max(0LL, atoll(v));
    w->prof = &ctx->prof;
    *out = std::move(w);
    return PGET_OK;
}

// The workspace of the direct (non-serving) calls: reused while the geometry and
// precision stay the same; counted against the budget together with serving slots.
pget_status get_workspace(pget_ctx* ctx, const pget_geometry* gin, int prec, Workspace** out) {
    Geometry g;
    std::string key;
    int groups = 1;
    size_t need = 0;
    pget_status s = resolve(gin, prec, &g, &key, &groups, &need);
    if (s != PGET_OK) return s;
    if (ctx->ws && ctx->ws_key == key) {
        *out = ctx->ws.get();
        return PGET_OK;
    }
    if (ctx->budget)  // idle serving workspaces give way to the direct path
        while (need + serving_bytes(ctx) > ctx->budget && evict_idle(ctx)) {
        }
    if (ctx->budget && need + serving_bytes(ctx) > ctx->budget)
        return fail(PGET_ENOMEM, "workspace needs %zu bytes, budget %zu (serving slots hold %zu)", need,
                    ctx->budget, serving_bytes(ctx));
    ctx->ws.reset();
    ctx->ws_key.clear();
    std::unique_ptr<Workspace> w;
    s = make_workspace(ctx, std::move(g), prec, groups, &w);
    if (s != PGET_OK) return s;
    ctx->ws = std::move(w);
    ctx->ws_key = key;
    *out = ctx->ws.get();
    return PGET_OK;
}

// ------------------------------------------------------------------ operators
WalkArgs base_args(const Workspace& w) {
    WalkArgs a{};
    const Geometry& G = w.g;
    a.views = w.d_views;
    a.n = G.n;
    a.T = G.T;
    a.P = w.P;
    a.h = G.h;
    a.max_slots = G.max_slots;
    a.n_det = G.n_det;
    a.n_banks = G.n_banks;
    a.nb = G.nb;
    a.n_sub = G.n_sub;
    a.det_slot = w.d_det_slot;
    a.w = w.d_w;
    a.src_off = w.d_src_off;
    a.src_det = w.d_src_det;
    a.src_w = w.d_src_w;
    a.clip = w.d_clip;
    a.depth = w.d_depth;
    a.err = w.err;
    a.tx_extra = w.tx_extra;
    a.wait_ns = w.wait_ns;
    a.cta_order = w.d_view_order;  // views; the adjoint launches replace it by the group order
    return a;
}

cudaError_t op_forward(const Workspace& w, void* const pk[2], void* U_out, void* y_out, const int* stop, cudaStream_t st) {
    WalkArgs a = base_args(w);
    a.Yc = w.pf.Yc;
    a.nchunks = w.pf.nchunks;
    a.u_img[0] = pk[0];
    a.u_img[1] = pk[1];
    a.slot_val = U_out;
    a.y_out = w.sino_w ? w.sino_w : y_out;  // a sinogram in the walks' type, widened below
    a.stop = stop;
    w.prof->begin(kPFwd, st);
    cudaError_t e = launch_walk(kFwd, w.wprec, w.pf, a, w.n_views, st);
    w.prof->end(st);
    if (e == cudaSuccess && w.sino_w) convert<float, double>((const float*)w.sino_w, (double*)y_out, w.M, stop, st);
    return e;
}

cudaError_t op_jvp(const Workspace& w, void* const pku[2], void* const pkp[2], void* dy, const int* stop, cudaStream_t st) {
    WalkArgs a = base_args(w);
    a.Yc = w.pj.Yc;
    a.nchunks = w.pj.nchunks;
    a.u_img[0] = pku[0];
    a.u_img[1] = pku[1];
    a.p_img[0] = pkp[0];
    a.p_img[1] = pkp[1];
    a.y_out = w.sino_w ? w.sino_w : dy;
    a.stop = stop;
    w.prof->begin(kPJvp, st);
    cudaError_t e = launch_walk(kJvp, w.wprec, w.pj, a, w.n_views, st);
    w.prof->end(st);
    if (e == cudaSuccess && w.sino_w) convert<float, double>((const float*)w.sino_w, (double*)dy, w.M, stop, st);
    return e;
}

// The forward model at the planar point uvec (solver type), whose walk layouts pk the
// caller has packed, where its value enters the objective: op_forward, except in
// PGET_MIXED, where it runs in double (own layouts and plan) straight into the double
// sinogram y_out, and the ray totals are narrowed to the float ones the adjoint reads.
cudaError_t op_objective(Workspace& w, const void* uvec, void* const pk[2], void* U_out, void* y_out,
                         const int* stop, cudaStream_t st) {
    if (!w.obj64) return op_forward(w, pk, U_out, y_out, stop, st);
    const double* u = (const double*)uvec;
    pack<double, double>(u, u + w.nn, w.g.n, w.P, attenuation_scale(w.g), w.pk64[0], w.pk64[1], stop, st);
    WalkArgs a = base_args(w);
    a.w = w.d_w64;
    a.depth = w.d_depth64;
    a.Yc = w.pf64.Yc;
    a.nchunks = w.pf64.nchunks;
    a.u_img[0] = w.pk64[0];
    a.u_img[1] = w.pk64[1];
    a.slot_val = U_out ? w.U64 : nullptr;
    a.y_out = y_out;
    a.stop = stop;
    w.prof->begin(kPFwd, st);
    cudaError_t e = launch_walk(kFwd, PGET_F64, w.pf64, a, w.n_views, st);
    w.prof->end(st);
    if (e == cudaSuccess && U_out) convert<double, float>((const double*)w.U64, (float*)U_out, w.nslots, stop, st);
    return e;
}

// J^T r (+ optional prior / damping / dot through ra)
template <typename T>
cudaError_t op_vjp(Workspace& w, void* const pku[2], const void* U, const void* r, RedArgs<T> ra,
                   const int* stop, cudaStream_t st) {
    WalkArgs a = base_args(w);
    a.Yc = w.pv.Yc;
    a.nchunks = w.pv.nchunks;
    a.sb_cap = w.pv.sb_cap;
    a.u_img[0] = pku[0];
    a.u_img[1] = pku[1];
    a.slot_val = (void*)U;
    a.r_in = r;
    if (w.sino_w) {  // the residual in the walks' type
        convert<double, float>((const double*)r, (float*)w.sino_w, w.M, stop, st);
        a.r_in = w.sino_w;
    }
    a.gpart = w.gpart;
    a.win = w.d_win;
    a.group_off = w.d_group_off;
    a.group_view = w.d_group_view;
    a.cta_order = w.d_group_order;
    a.stop = stop;
    w.prof->begin(kPVjp, st);
    cudaError_t e = launch_walk(kVjp, w.wprec, w.pv, a, w.n_groups, st);
    w.prof->end(st);
    if (e != cudaSuccess) return e;
    ra.n = w.g.n;
    ra.skip = stop;
    w.prof->begin(kPRed, st);
    // the view sum is already two-level (<= ~40 terms per level): plain sums suffice;
    // the Kahan compensation of PGET_F32_KAHAN applies along rays
    if (w.wf64 || sizeof(T) == 4)
        reduce_views<T, T>((const T*)w.gpart, w.g.n, w.n_groups, w.n_groups0, w.groups, (T*)w.part2, ra, false, st);
    else
        reduce_views<T, float>((const float*)w.gpart, w.g.n, w.n_groups, w.n_groups0, w.groups, (float*)w.part2, ra,
                               false, st);
    w.prof->end(st);
    return cudaGetLastError();
}

// planar solver vectors (type T) -> the walks' packed layouts (their own type)
template <typename T>
void pack_pair(const Workspace& w, const void* lam, const void* mu, void* const pk[2], const int* skip,
               cudaStream_t st) {
    const T* l = (const T*)lam;
    const T* m = (const T*)mu;
    if (w.wf64 || sizeof(T) == 4) pack<T, T>(l, m, w.g.n, w.P, attenuation_scale(w.g), pk[0], pk[1], skip, st);
    else pack<T, float>(l, m, w.g.n, w.P, attenuation_scale(w.g), pk[0], pk[1], skip, st);
}

template <typename T>
void pack_vec(const Workspace& w, const void* vec, void* const pk[2], const int* skip, cudaStream_t st) {
    pack_pair<T>(w, vec, (const T*)vec + w.nn, pk, skip, st);
}

template <typename T>
void pack_pair(const Workspace& w, const void* lam, const void* mu, void* const pk[2], cudaStream_t st) {
    pack_pair<T>(w, lam, mu, pk, nullptr, st);
}

// Geometry priors of Eq. (6) in a fused reduction: the Hessian term (gradient = false) or
// the gradient 2 alpha (1 - M)^2 (u - c) (gradient = true, c = mu_water on the mu field).
template <typename T>
void set_geo(RedArgs<T>& a, const pget_lm_params& p, bool gradient) {
    a.gmask = (const T*)p.geo_mask;
    a.geo_l = p.geo_alpha_lambda;
    a.geo_m = p.geo_alpha_mu;
    a.geo_cm = p.geo_mu_water;
    a.geo_offset = gradient ? 1 : 0;
}

// CG on (J^T J + H + nu I) x = scale_b * b, H and U at the packed iterate pk_u
template <typename T>
pget_status run_cg(Workspace& w, const void* b, double scale_b, double nu, const double* nu_dev,
                   const pget_lm_params& p, cudaStream_t st) {
    const size_t m = 2 * w.nn;
    CgState* cg = &w.lm->cg;
    cg_init<T>((const T*)b, (T*)w.x, (T*)w.res, (T*)w.p, m, scale_b, p.cg_rel_tol, w.dpart[0], cg, st);
    const int* stop = &cg->stop;
    pack_vec<T>(w, w.p, w.pk_p, stop, st);  // later directions are packed by cg_dir_pack
    for (int it = 0; it < p.cg_max_iters; ++it) {
        cudaError_t e = op_jvp(w, w.pk_u, w.pk_p, w.Jp, stop, st);
        if (e != cudaSuccess) return fail(PGET_ECUDA, "jvp launch: %s", cudaGetErrorString(e));
        RedArgs<T> ra;
        ra.out = (T*)w.q;
        ra.v = (const T*)w.p;
        ra.Wl = (const T*)w.Wl;
        ra.Wm = (const T*)w.Wm;
        ra.alpha_l = p.alpha_lambda;
        ra.alpha_m = p.alpha_mu;
        set_geo(ra, p, false);
        ra.nu = nu;
        ra.nu_dev = nu_dev;
        ra.dotv = (const T*)w.p;
        ra.part = w.dpart[0];
        e = op_vjp<T>(w, w.pk_u, w.U, w.Jp, ra, stop, st);
        if (e != cudaSuccess) return fail(PGET_ECUDA, "vjp launch: %s", cudaGetErrorString(e));
        cg_step<T>((T*)w.x, (T*)w.res, (const T*)w.p, (const T*)w.q, m, w.dpart[0], w.dpart[1], cg, st);
        if (w.wf64 || sizeof(T) == 4)
            cg_dir_pack<T, T>((T*)w.p, (const T*)w.res, w.dpart[1], cg, w.g.n, w.P, attenuation_scale(w.g), w.pk_p[0],
                              w.pk_p[1], st);
        else
            cg_dir_pack<T, float>((T*)w.p, (const T*)w.res, w.dpart[1], cg, w.g.n, w.P, attenuation_scale(w.g),
                                  w.pk_p[0], w.pk_p[1], st);
    }
    CK(cudaGetLastError());
    return PGET_OK;
}

// device error flags: bit 1 an adjoint stencil bound was violated (never expected: the
// geometry guarantees it), bit 2 a chunk copy did not complete within the wait limit
pget_status flags_status(int e) {
    if (e & 4) return fail(PGET_ETIMEOUT, "device error flags 0x%x (chunk copy wait timed out)", e);
    if (e) return fail(PGET_ECUDA, "device error flags 0x%x (adjoint stencil bound)", e);
    return PGET_OK;
}

// the constraint set of the parameters: the box and the optional linear bound
static Feas feas_of(const pget_lm_params& p) {
    return make_feas(p.lambda_max, p.mu_max, p.lin_constraint, p.lin_slope, p.lin_offset);
}

// Gradient projection on min <g, s> + 1/2 s^T (J^T J + H + nu I) s subject to u + s in the
// constraint set, u the unpacked iterate in w.u (packed in pk_u), g in gvec; result
// (feasible) in w.x.
// One J^T J product per iteration, like a CG step; the scalars live in w.lm->cg.
template <typename T>
pget_status run_sgp(Workspace& w, const void* gvec, double nu, const double* nu_dev, const pget_lm_params& p,
                    cudaStream_t st) {
    const size_t nn = w.nn, m = 2 * nn;
    CgState* cg = &w.lm->cg;
    sgp_init<T>((const T*)gvec, (T*)w.res, (T*)w.x, m, p.cg_rel_tol, cg, st);
    const int* stop = &cg->stop;
    for (int it = 0; it < p.cg_max_iters; ++it) {
        sgp_dir<T>((const T*)w.u, (const T*)w.x, (const T*)w.res, (T*)w.p, nn, feas_of(p), w.dpart[1],
                   w.dpart[2], w.dpart[3], cg, st);
        pack_vec<T>(w, w.p, w.pk_p, stop, st);
        cudaError_t e = op_jvp(w, w.pk_u, w.pk_p, w.Jp, stop, st);
        if (e != cudaSuccess) return fail(PGET_ECUDA, "jvp launch: %s", cudaGetErrorString(e));
        RedArgs<T> ra;
        ra.out = (T*)w.q;
        ra.v = (const T*)w.p;
        ra.Wl = (const T*)w.Wl;
        ra.Wm = (const T*)w.Wm;
        ra.alpha_l = p.alpha_lambda;
        ra.alpha_m = p.alpha_mu;
        set_geo(ra, p, false);
        ra.nu = nu;
        ra.nu_dev = nu_dev;
        ra.dotv = (const T*)w.p;
        ra.part = w.dpart[0];
        e = op_vjp<T>(w, w.pk_u, w.U, w.Jp, ra, stop, st);
        if (e != cudaSuccess) return fail(PGET_ECUDA, "vjp launch: %s", cudaGetErrorString(e));
        dot<T>((const T*)w.q, (const T*)w.q, m, w.dpart[1], stop, st);
        sgp_step(w.dpart[0], w.dpart[1], cg, st);
        sgp_update<T>((T*)w.x, (T*)w.res, (const T*)w.p, (const T*)w.q, m, cg, st);
    }
    CK(cudaGetLastError());
    return PGET_OK;
}

pget_status check_err(Workspace& w, cudaStream_t st) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return flags_status(e);
}

void params_dev(const pget_lm_params& p, LmParamsDev* d) {
    d->eta = p.eta;
    d->rho_lo = p.rho_lo;
    d->rho_hi = p.rho_hi;
    d->nu_up = p.nu_up;
    d->nu_down = p.nu_down;
    d->nu_min = p.nu_min;
    d->nu_max = p.nu_max;
}

pget_status check_params(const pget_lm_params* p) {
    if (!p) return fail(PGET_EINVAL, "null params");
    if (p->max_iters < 0 || p->cg_max_iters < 0) return fail(PGET_EINVAL, "negative iteration count");
    if (!(p->lambda_max > 0) || !(p->mu_max > 0)) return fail(PGET_EINVAL, "box bounds must be positive");
    if (!(p->alpha_lambda >= 0) || !(p->alpha_mu >= 0)) return fail(PGET_EINVAL, "prior weights must be >= 0");
    if (!(p->nu_up >= 1) || !(p->nu_down > 0 && p->nu_down <= 1)) return fail(PGET_EINVAL, "bad nu_up / nu_down");
    if (!std::isfinite(p->tv_eps)) return fail(PGET_EINVAL, "tv_eps must be finite (<= 0: quadratic prior)");
    if (std::isnan(p->cg_rel_tol)) return fail(PGET_EINVAL, "cg_rel_tol is NaN");
    if (!(p->nu0_scale > 0) || !std::isfinite(p->nu0_scale)) return fail(PGET_EINVAL, "nu0_scale must be finite and > 0");
    if (!std::isfinite(p->eta) || !std::isfinite(p->rho_lo) || !std::isfinite(p->rho_hi) || !(p->rho_lo <= p->rho_hi))
        return fail(PGET_EINVAL, "eta, rho_lo and rho_hi must be finite, rho_lo <= rho_hi");
    if (!(p->nu_min > 0) || !(p->nu_min <= p->nu_max)) return fail(PGET_EINVAL, "need 0 < nu_min <= nu_max");
    if (!known_precision(p->precision)) return fail(PGET_EINVAL, "unknown precision %d", p->precision);
    if (!(p->alpha_decay == 0.0 || p->alpha_decay >= 1.0) || p->alpha_decay_iters < 0)
        return fail(PGET_EINVAL, "alpha_decay must be 0 or >= 1 and alpha_decay_iters >= 0");
    if (p->geo_mask && (!(p->geo_alpha_lambda >= 0) || !(p->geo_alpha_mu >= 0) || !std::isfinite(p->geo_mu_water)))
        return fail(PGET_EINVAL, "geometry prior weights must be >= 0");
    if (p->inner_solver != 0 && p->inner_solver != 1) return fail(PGET_EINVAL, "inner_solver must be 0 or 1");
    if (p->lin_constraint != 0 && p->lin_constraint != 1) return fail(PGET_EINVAL, "lin_constraint must be 0 or 1");
    if (p->lin_constraint && !(p->lin_slope >= 0.0 && std::isfinite(p->lin_slope) && p->lin_offset >= 0.0 &&
                               std::isfinite(p->lin_offset)))
        return fail(PGET_EINVAL, "linear bound: lin_slope and lin_offset must be finite and >= 0");
    return PGET_OK;
}

// Prior weights of LM iteration k under the continuation of Sec. 3.1:
// alpha / alpha_decay^min(k, alpha_decay_iters) (fixed when alpha_decay <= 1 or no iterations).
pget_lm_params params_at(const pget_lm_params& p, int k) {
    pget_lm_params q = p;
    if (p.alpha_decay > 1.0 && p.alpha_decay_iters > 0) {
        const double sc = std::pow(p.alpha_decay, -(double)std::min(k, p.alpha_decay_iters));
        q.alpha_lambda *= sc;
        q.alpha_mu *= sc;
        q.geo_alpha_lambda *= sc;
        q.geo_alpha_mu *= sc;
    }
    return q;
}

// LM solve on device pointers (y, u0 planar inputs copied into the workspace)
// The LM iteration proper: reads yb and the initial guess in u, leaves the result in u
// and the scalars and traces in w.lm.  Only kernel launches (no host synchronisation),
// so it can be captured as a CUDA graph.
template <typename T>
pget_status lm_body(Workspace& w, const pget_lm_params& p, cudaStream_t st) {
    const size_t nn = w.nn, M = w.M;
    const int n = w.g.n;
    LmState* L = w.lm;
    project_set<T>((T*)w.u, nn, feas_of(p), st);
    pack_vec<T>(w, w.u, w.pk_u, nullptr, st);
    T* u = (T*)w.u;
    // objective and gradient at u_0
    CK(op_objective(w, w.u, w.pk_u, w.U, w.Jp, nullptr, st));
    sub_dot<T>((const T*)w.Jp, (const T*)w.yb, (T*)w.r, M, w.dpart[0], nullptr, st);
    finish_sum(w.dpart[0], &L->rtrt, nullptr, st);
    reg_value<T>(u, n, p.alpha_lambda, p.tv_eps, w.dpart[1], nullptr, st, (const T*)p.geo_mask, p.geo_alpha_lambda, 0.0);
    finish_sum(w.dpart[1], &L->Rl, nullptr, st);
    reg_value<T>(u + nn, n, p.alpha_mu, p.tv_eps, w.dpart[2], nullptr, st, (const T*)p.geo_mask, p.geo_alpha_mu, p.geo_mu_water);
    finish_sum(w.dpart[2], &L->Rm, nullptr, st);
    reg_weights<T>(u, n, p.tv_eps, (T*)w.Wl, nullptr, st);
    reg_weights<T>(u + nn, n, p.tv_eps, (T*)w.Wm, nullptr, st);
    RedArgs<T> ga;
    ga.out = (T*)w.gr;
    ga.v = u;
    ga.Wl = (const T*)w.Wl;
    ga.Wm = (const T*)w.Wm;
    ga.alpha_l = p.alpha_lambda;
    ga.alpha_m = p.alpha_mu;
    set_geo(ga, p, true);
    ga.nu = 0.0;
    CK(op_vjp<T>(w, w.pk_u, w.U, w.r, ga, nullptr, st));
    dot<T>((const T*)w.gr, (const T*)w.gr, 2 * nn, w.dpart[0], nullptr, st);
    finish_sum(w.dpart[0], &L->gg, nullptr, st);
    pack_vec<T>(w, w.gr, w.pk_p, nullptr, st);
    CK(op_jvp(w, w.pk_u, w.pk_p, w.Jp, nullptr, st));
    dot<T>((const T*)w.Jp, (const T*)w.Jp, M, w.dpart[0], nullptr, st);
    finish_sum(w.dpart[0], &L->JsJs, nullptr, st);
    lm_init_f(L, p.nu0_scale, st);
    LmParamsDev pd;
    params_dev(p, &pd);
    const int* no_grad = &L->no_grad;
    pget_lm_params pk = params_at(p, 0);
    for (int k = 0; k < p.max_iters; ++k) {
        // continuation: new prior weights change f and its gradient at the current iterate
        const pget_lm_params nk = params_at(p, k);
        const bool refresh = k > 0 && (nk.alpha_lambda != pk.alpha_lambda || nk.alpha_mu != pk.alpha_mu);
        pk = nk;
        ga.alpha_l = pk.alpha_lambda;
        ga.alpha_m = pk.alpha_mu;
        set_geo(ga, pk, true);
        if (refresh) {
            dot<T>((const T*)w.r, (const T*)w.r, M, w.dpart[0], nullptr, st);
            finish_sum(w.dpart[0], &L->rtrt, nullptr, st);
            reg_value<T>(u, n, pk.alpha_lambda, pk.tv_eps, w.dpart[1], nullptr, st, (const T*)pk.geo_mask, pk.geo_alpha_lambda, 0.0);
            finish_sum(w.dpart[1], &L->Rl, nullptr, st);
            reg_value<T>(u + nn, n, pk.alpha_mu, pk.tv_eps, w.dpart[2], nullptr, st, (const T*)pk.geo_mask, pk.geo_alpha_mu, pk.geo_mu_water);
            finish_sum(w.dpart[2], &L->Rm, nullptr, st);
            lm_refresh_f(L, st);
        }
        const int* skip_grad = refresh ? nullptr : no_grad;
        // gradient and prior weights at a newly accepted iterate
        reg_weights<T>(u, n, p.tv_eps, (T*)w.Wl, skip_grad, st);
        reg_weights<T>(u + nn, n, p.tv_eps, (T*)w.Wm, skip_grad, st);
        CK(op_vjp<T>(w, w.pk_u, w.U, w.r, ga, skip_grad, st));
        // step from the damped normal equations, rhs = -grad
        pget_status s = pk.inner_solver == 1 ? run_sgp<T>(w, w.gr, 0.0, &L->nu, pk, st)
                                             : run_cg<T>(w, w.gr, -1.0, 0.0, &L->nu, pk, st);
        if (s != PGET_OK) return s;
        lm_step<T>(u, (const T*)w.x, (T*)w.ut, (T*)w.s, nn, feas_of(p), st);
        pack_vec<T>(w, w.ut, w.pk_ut, nullptr, st);
        pack_vec<T>(w, w.s, w.pk_p, nullptr, st);
        lm_model<T>((const T*)w.s, (const T*)w.gr, (const T*)w.Wl, (const T*)w.Wm, n, pk.alpha_lambda,
                    pk.alpha_mu, w.dpart[0], w.dpart[1], st, (const T*)pk.geo_mask, pk.geo_alpha_lambda, pk.geo_alpha_mu);
        finish_sum(w.dpart[0], &L->sg, nullptr, st);
        finish_sum(w.dpart[1], &L->sHs, nullptr, st);
        CK(op_jvp(w, w.pk_u, w.pk_p, w.Jp, nullptr, st));
        dot<T>((const T*)w.Jp, (const T*)w.Jp, M, w.dpart[2], nullptr, st);
        finish_sum(w.dpart[2], &L->JsJs, nullptr, st);
        CK(op_objective(w, w.ut, w.pk_ut, w.Ut, w.rt, nullptr, st));
        sub_dot<T>((const T*)w.rt, (const T*)w.yb, (T*)w.rt, M, w.dpart[3], nullptr, st);
        finish_sum(w.dpart[3], &L->rtrt, nullptr, st);
        const T* ut = (const T*)w.ut;
        reg_value<T>(ut, n, pk.alpha_lambda, pk.tv_eps, w.dpart[1], nullptr, st, (const T*)pk.geo_mask, pk.geo_alpha_lambda, 0.0);
        finish_sum(w.dpart[1], &L->Rl, nullptr, st);
        reg_value<T>(ut + nn, n, pk.alpha_mu, pk.tv_eps, w.dpart[2], nullptr, st, (const T*)pk.geo_mask, pk.geo_alpha_mu, pk.geo_mu_water);
        finish_sum(w.dpart[2], &L->Rm, nullptr, st);
        lm_decide(L, pd, st);
        const int* acc = &L->accept;
        copy_if<T>((T*)w.u, ut, 2 * nn, acc, st);
        copy_if<T>((T*)w.r, (const T*)w.rt, M, acc, st);
        if (w.wf64) copy_if<double>((double*)w.U, (const double*)w.Ut, w.nslots, acc, st);
        else copy_if<float>((float*)w.U, (const float*)w.Ut, w.nslots, acc, st);
        if (w.wf64) {
            copy_if<double2>((double2*)w.pk_u[0], (const double2*)w.pk_ut[0], w.img_elems, acc, st);
            copy_if<double2>((double2*)w.pk_u[1], (const double2*)w.pk_ut[1], w.img_elems, acc, st);
        } else {
            copy_if<float2>((float2*)w.pk_u[0], (const float2*)w.pk_ut[0], w.img_elems, acc, st);
            copy_if<float2>((float2*)w.pk_u[1], (const float2*)w.pk_ut[1], w.img_elems, acc, st);
        }
        CK(cudaGetLastError());
    }
    return PGET_OK;
}

// key of a captured LM graph: every parameter baked into its kernels
static std::string graph_key(const pget_lm_params& p, bool prof) {
    std::string k((const char*)&p, sizeof p);
    k += prof ? "P" : "N";
    return k;
}

// Enqueue one LM solve on st: yb and the initial guess in u must already be in the
// workspace.  The body runs as a captured CUDA graph (replayed while the parameters stay
// the same); afterwards the device state and error flags are copied to pinned host
// memory.  Nothing here waits for the device.
template <typename T>
pget_status lm_launch(Workspace& w, const pget_lm_params& p, cudaStream_t st) {
    CK(cudaEventRecord(w.t0, st));
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    const char* ng = getenv("PGET_NO_GRAPH");
    const bool use_graph = !(ng && atoi(ng) > 0);
    if (use_graph) {
        const std::string key = graph_key(p, w.prof->on);
        if (!w.graph_exec || w.graph_key != key) {
            if (w.graph_exec) {
                cudaGraphExecDestroy(w.graph_exec);
                w.graph_exec = nullptr;
            }
            for (auto& r : w.graph_events) {
                cudaEventDestroy(r.a);
                cudaEventDestroy(r.b);
            }
            w.graph_events.clear();
            if (!w.cap_stream) CK(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking));
            CK(prepare_walk(kFwd, w.wprec, w.pf));
            CK(prepare_walk(kJvp, w.wprec, w.pj));
            CK(prepare_walk(kVjp, w.wprec, w.pv));
            if (w.obj64) CK(prepare_walk(kFwd, PGET_F64, w.pf64));
            const long long l0 = launch_count();
            CK(cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal));
            w.prof->capturing = true;
            pget_status bs = lm_body<T>(w, p, w.cap_stream);
            w.prof->capturing = false;
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(w.cap_stream, &graph);
            std::vector<Profiler::Rec> recs;
            recs.swap(w.prof->captured);
            if (bs != PGET_OK) {
                if (graph) cudaGraphDestroy(graph);
                return bs;
            }
            if (ce != cudaSuccess) return fail(PGET_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&w.graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                w.graph_exec = nullptr;
                return fail(PGET_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            }
            w.graph_key = key;
            w.graph_events = std::move(recs);
            w.graph_launches = launch_count() - l0;
        } else {
            note_launch((int)w.graph_launches);
        }
        CK(cudaGraphLaunch(w.graph_exec, st));
    } else {
        pget_status bs = lm_body<T>(w, p, st);
        if (bs != PGET_OK) return bs;
    }
    CK(cudaEventRecord(w.t1, st));
    CK(cudaMemcpyAsync(w.host_lm, w.lm, sizeof(LmState), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w.host_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    w.graph_used = use_graph;
    return PGET_OK;
}

// After the stream of an lm_launch has completed: profiler counters, error flags and
// the report (from the pinned copies).
pget_status lm_finish(Workspace& w, pget_lm_report* rep) {
    w.prof->collect();
    if (w.graph_used && w.prof->on) w.prof->collect_graph(w.graph_events);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w.t0, w.t1);
    if (*w.host_err) return flags_status(*w.host_err);
    const LmState* hl = w.host_lm;
    if (rep) {
        memset(rep, 0, sizeof *rep);
        rep->iters_run = hl->iter;
        rep->accepted = hl->accepted;
        rep->cg_iters_total = hl->cg_total;
        rep->f0 = hl->f0;
        rep->f_final = hl->f;
        rep->nu0 = hl->nu0;
        rep->nu_final = hl->nu;
        int kk = std::min(hl->iter, PGET_TRACE);
        for (int k = 0; k < kk; ++k) {
            rep->f[k] = hl->tr_f[k];
            rep->rho[k] = hl->tr_rho[k];
            rep->nu[k] = hl->tr_nu[k];
            rep->pred[k] = hl->tr_pred[k];
            rep->ared[k] = hl->tr_ared[k];
            rep->acc[k] = hl->tr_acc[k];
            rep->cg_iters[k] = hl->tr_cg[k];
        }
        rep->device_ms = ms;
        rep->status = std::isfinite(hl->f) ? PGET_OK : PGET_ENUMERIC;
    }
    if (!std::isfinite(hl->f)) return fail(PGET_ENUMERIC, "objective is not finite");
    return PGET_OK;
}

template <typename T>
pget_status lm_solve_impl(Workspace& w, const pget_lm_params& p, const void* y, const void* lam,
                          const void* mu, void* lam_out, void* mu_out, pget_lm_report* rep, cudaStream_t st) {
    const size_t nn = w.nn;
    if (y != w.yb) CK(cudaMemcpyAsync(w.yb, y, w.elt * w.M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(w.u, lam, w.elt * nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)w.u + w.elt * nn, mu, w.elt * nn, cudaMemcpyDeviceToDevice, st));
    pget_status s = lm_launch<T>(w, p, st);
    if (s != PGET_OK) return s;
    CK(cudaMemcpyAsync(lam_out, w.u, w.elt * nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(mu_out, (char*)w.u + w.elt * nn, w.elt * nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return lm_finish(w, rep);
}

size_t serving_bytes(const pget_ctx* ctx) {
    size_t b = 0;
    for (auto& sl : ctx->slots)
        if (sl->ws) b += sl->ws->bytes;
    for (auto& e : ctx->pool) b += e.ws->bytes;
    return b;
}

// Free the least recently used idle workspace; false when the pool is empty.
bool evict_idle(pget_ctx* ctx) {
    if (ctx->pool.empty()) return false;
    size_t k = 0;
    for (size_t i = 1; i < ctx->pool.size(); ++i)
        if (ctx->pool[i].last_use < ctx->pool[k].last_use) k = i;
    ctx->pool.erase(ctx->pool.begin() + k);
    return true;
}

// Memory the serving path may hold without a budget: a quarter of the device.
size_t default_serving_cap() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || tot == 0) return (size_t)8 << 30;
    return tot / 4;
}

// Initial guess on the device without host synchronisation (serving path): lambda is
// the constant c = sum y / sum A(1, mu0) (clamped to the box), mu = mu0.
template <typename T>
pget_status init_async(Workspace& w, const pget_lm_params& p, double mu_init, void* lam, void* mu, cudaStream_t st) {
    const size_t nn = w.nn;
    T* u = (T*)w.ut;
    fill<T>(u, nn, 1.0, st);
    const double mu0 = std::min(std::max(mu_init, 0.0), p.mu_max);
    fill<T>(u + nn, nn, mu0, st);
    pack_vec<T>(w, u, w.pk_ut, nullptr, st);
    CK(op_forward(w, w.pk_ut, nullptr, w.Jp, nullptr, st));
    fill<T>((T*)w.rt, w.M, 1.0, st);
    dot<T>((const T*)w.Jp, (const T*)w.rt, w.M, w.dpart[0], nullptr, st);
    finish_sum(w.dpart[0], &w.lm->init_sa, nullptr, st);
    dot<T>((const T*)w.yb, (const T*)w.rt, w.M, w.dpart[1], nullptr, st);
    finish_sum(w.dpart[1], &w.lm->init_sy, nullptr, st);
    fill_ratio<T>((T*)lam, nn, &w.lm->init_sy, &w.lm->init_sa, p.lambda_max, st);
    fill<T>((T*)mu, nn, mu0, st);
    CK(cudaGetLastError());
    return PGET_OK;
}

int max_inflight() {
    const char* v = getenv("PGET_MAX_INFLIGHT");
    int k = v ? atoi(v) : 0;
    return k > 0 ? std::min(k, 64) : 8;
}

}  // namespace

// ========================================================================= C ABI
namespace {

template <typename T>
static pget_status vjp_impl(Workspace& w, const void* lam, const void* mu, const void* r, void* gl, void* gm,
                            cudaStream_t st) {
    pack_pair<T>(w, lam, mu, w.pk_u, st);
    CK(op_forward(w, w.pk_u, w.U, w.Jp, nullptr, st));
    RedArgs<T> ra;
    ra.out = (T*)w.q;
    CK(op_vjp<T>(w, w.pk_u, w.U, r, ra, nullptr, st));
    CK(cudaMemcpyAsync(gl, w.q, w.elt * w.nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(gm, (char*)w.q + w.elt * w.nn, w.elt * w.nn, cudaMemcpyDeviceToDevice, st));
    return PGET_OK;
}

// Buffers for chunks of up to B items of workspace w (reallocated when the workspace or
// the chunk size changes); *cap gets the items per chunk.
static pget_status get_batch(pget_ctx* ctx, Workspace& w, int B, BatchBufs** out) {
    const long long s_img = (long long)(2 * w.welt * w.img_elems);
    const long long s_slot = (long long)(w.welt * w.nslots), s_sino = (long long)(w.welt * w.M);
    const long long s_part = (long long)(w.welt * (size_t)w.n_groups * 2 * w.nn);
    int cap = (int)std::max<long long>(1, std::min<long long>(B, (long long)kBatchPartBytes / std::max(1LL, s_part)));
    BatchBufs* bb = ctx->batch.get();
    if (bb && bb->key == ctx->ws_key && bb->cap >= cap) {
        *out = bb;
        return PGET_OK;
    }
    ctx->batch.reset();
    auto nb = std::make_unique<BatchBufs>();
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) {
            nb->allocs.push_back(*p);
            e = cudaMemset(*p, 0, bytes ? bytes : 16);  // zero borders of the packed layouts
        }
        return e;
    };
    for (int l = 0; l < 2; ++l) {
        CK(alloc(&nb->pk_u[l], (size_t)s_img * cap));
        CK(alloc(&nb->pk_p[l], (size_t)s_img * cap));
    }
    CK(alloc(&nb->U, (size_t)s_slot * cap));
    CK(alloc(&nb->sino, (size_t)s_sino * cap));
    CK(alloc(&nb->gpart, (size_t)s_part * cap));
    nb->key = ctx->ws_key;
    nb->cap = cap;
    nb->s_img = s_img;
    nb->s_slot = s_slot;
    nb->s_sino = s_sino;
    nb->s_part = s_part;
    ctx->batch = std::move(nb);
    *out = ctx->batch.get();
    return PGET_OK;
}

// the layouts of item k of a chunk
static void item_layouts(void* const base[2], long long stride, int k, void* out[2]) {
    out[0] = (char*)base[0] + stride * k;
    out[1] = (char*)base[1] + stride * k;
}

// mode kFwd: y = A(lam, mu); kJvp: y = J (dl, dm); kVjp: (gl, gm) = J^T r, for `batch`
// items stored one after another, in chunks of bb->cap items per walk launch.  Every
// item's result equals the single-item call's bitwise (same kernels and plans).
template <typename T>
static pget_status batch_impl(pget_ctx* ctx, Workspace& w, int mode, int batch, const void* lam, const void* mu,
                              const void* dl, const void* dm, const void* r, void* y, void* gl, void* gm,
                              cudaStream_t st) {
    BatchBufs* bb;
    pget_status s = get_batch(ctx, w, batch, &bb);
    if (s != PGET_OK) return s;
    const size_t nn = w.nn, e = w.elt;
    for (int i0 = 0; i0 < batch; i0 += bb->cap) {
        const int b = std::min(bb->cap, batch - i0);
        for (int k = 0; k < b; ++k) {
            void* pu[2];
            item_layouts(bb->pk_u, bb->s_img, k, pu);
            pack_pair<T>(w, (const char*)lam + e * nn * (i0 + k), (const char*)mu + e * nn * (i0 + k), pu, st);
            if (mode == kJvp) {
                void* pp[2];
                item_layouts(bb->pk_p, bb->s_img, k, pp);
                pack_pair<T>(w, (const char*)dl + e * nn * (i0 + k), (const char*)dm + e * nn * (i0 + k), pp, st);
            }
        }
        WalkArgs a = base_args(w);
        a.u_img[0] = bb->pk_u[0];
        a.u_img[1] = bb->pk_u[1];
        a.n_items = b;
        a.s_img = bb->s_img;
        a.s_sino = bb->s_sino;
        a.s_slot = bb->s_slot;
        a.s_part = bb->s_part;
        cudaError_t ce;
        if (mode == kJvp) {
            a.Yc = w.pj.Yc;
            a.nchunks = w.pj.nchunks;
            a.p_img[0] = bb->pk_p[0];
            a.p_img[1] = bb->pk_p[1];
            a.y_out = (char*)y + e * w.M * i0;
            w.prof->begin(kPJvp, st);
            ce = launch_walk(kJvp, w.wprec, w.pj, a, w.n_views, st);
            w.prof->end(st);
            CK(ce);
            continue;
        }
        // forward: into y, or (adjoint) into the scratch sinograms with the ray totals
        a.Yc = w.pf.Yc;
        a.nchunks = w.pf.nchunks;
        a.y_out = mode == kFwd ? (char*)y + e * w.M * i0 : bb->sino;
        a.slot_val = mode == kFwd ? nullptr : bb->U;
        w.prof->begin(kPFwd, st);
        ce = launch_walk(kFwd, w.wprec, w.pf, a, w.n_views, st);
        w.prof->end(st);
        CK(ce);
        if (mode == kFwd) continue;
        a.Yc = w.pv.Yc;
        a.nchunks = w.pv.nchunks;
        a.y_out = nullptr;
        a.slot_val = bb->U;
        a.r_in = (const char*)r + e * w.M * i0;
        a.gpart = bb->gpart;
        a.win = w.d_win;
        a.group_off = w.d_group_off;
        a.group_view = w.d_group_view;
        a.cta_order = w.d_group_order;
        w.prof->begin(kPVjp, st);
        ce = launch_walk(kVjp, w.wprec, w.pv, a, w.n_groups, st);
        w.prof->end(st);
        CK(ce);
        for (int k = 0; k < b; ++k) {  // the view sum of every item, as pget_vjp forms it
            RedArgs<T> ra;
            ra.out = (T*)w.q;
            ra.n = w.g.n;
            w.prof->begin(kPRed, st);
            reduce_views<T, T>((const T*)((const char*)bb->gpart + bb->s_part * k), w.g.n, w.n_groups, w.n_groups0,
                               w.groups, (T*)w.part2, ra, false, st);
            w.prof->end(st);
            CK(cudaMemcpyAsync((char*)gl + e * nn * (i0 + k), w.q, e * nn, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync((char*)gm + e * nn * (i0 + k), (char*)w.q + e * nn, e * nn, cudaMemcpyDeviceToDevice,
                               st));
        }
    }
    CK(cudaGetLastError());
    return PGET_OK;
}

template <typename T>
static pget_status cg_impl(Workspace& w, const pget_lm_params& p, const void* lam, const void* mu, double nu,
                           const void* rhs, void* x, int32_t* iters, cudaStream_t st) {
    const int n = w.g.n;
    pack_pair<T>(w, lam, mu, w.pk_u, st);
    CK(op_forward(w, w.pk_u, w.U, w.Jp, nullptr, st));
    reg_weights<T>((const T*)lam, n, p.tv_eps, (T*)w.Wl, nullptr, st);
    reg_weights<T>((const T*)mu, n, p.tv_eps, (T*)w.Wm, nullptr, st);
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    pget_status s = run_cg<T>(w, rhs, 1.0, nu, nullptr, p, st);
    if (s != PGET_OK) return s;
    CK(cudaMemcpyAsync(x, w.x, w.elt * 2 * w.nn, cudaMemcpyDeviceToDevice, st));
    if (iters) {
        CgState hc;
        CK(cudaMemcpyAsync(&hc, &w.lm->cg, sizeof hc, cudaMemcpyDeviceToHost, st));
        s = check_err(w, st);
        if (s != PGET_OK) return s;
        *iters = hc.iters;
    }
    return PGET_OK;
}

// FP64 block partials (kRedBlocks each) -> sums, finished on the host in a fixed order
static pget_status host_sums(Workspace& w, std::initializer_list<const double*> parts, double* out,
                             cudaStream_t st) {
    std::vector<double> h(parts.size() * kRedBlocks);
    size_t k = 0;
    for (const double* p : parts)
        CK(cudaMemcpyAsync(h.data() + kRedBlocks * k++, p, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t j = 0; j < parts.size(); ++j) {
        double a = 0.0;
        for (int b = 0; b < kRedBlocks; ++b) a += h[j * kRedBlocks + b];
        out[j] = a;
    }
    return PGET_OK;
}

// Objective f(u) = 1/2 |A(u) - y|^2 + R_lambda + R_mu at the packed point pk (u planar in
// uvec); leaves the residual A(u) - y in r and the ray totals in U.
template <typename T>
static pget_status objective_at(Workspace& w, const pget_lm_params& p, void* const pk[2], const void* uvec,
                                void* U, void* r, double* f, cudaStream_t st) {
    const T* u = (const T*)uvec;
    CK(op_objective(w, uvec, pk, U, w.Jp, nullptr, st));
    sub_dot<T>((const T*)w.Jp, (const T*)w.yb, (T*)r, w.M, w.dpart[0], nullptr, st);
    reg_value<T>(u, w.g.n, p.alpha_lambda, p.tv_eps, w.dpart[1], nullptr, st, (const T*)p.geo_mask, p.geo_alpha_lambda, 0.0);
    reg_value<T>(u + w.nn, w.g.n, p.alpha_mu, p.tv_eps, w.dpart[2], nullptr, st, (const T*)p.geo_mask, p.geo_alpha_mu, p.geo_mu_water);
    double v[3];
    pget_status s = host_sums(w, {w.dpart[0], w.dpart[1], w.dpart[2]}, v, st);
    if (s != PGET_OK) return s;
    *f = 0.5 * v[0] + v[1] + v[2];
    return PGET_OK;
}

// m_k(0) - m_k(s) at the packed iterate for the planar step s (gradient in w.gr, prior
// weights in Wl, Wm): -<s, g> - |J s|^2 / 2 - s^T H s / 2 (Eq. (8)).
template <typename T>
static pget_status model_decrease(Workspace& w, const pget_lm_params& p, const void* s, double* pred,
                                  cudaStream_t st) {
    lm_model<T>((const T*)s, (const T*)w.gr, (const T*)w.Wl, (const T*)w.Wm, w.g.n, p.alpha_lambda, p.alpha_mu,
                w.dpart[0], w.dpart[1], st, (const T*)p.geo_mask, p.geo_alpha_lambda, p.geo_alpha_mu);
    pack_vec<T>(w, s, w.pk_p, nullptr, st);
    CK(op_jvp(w, w.pk_u, w.pk_p, w.Jp, nullptr, st));
    dot<T>((const T*)w.Jp, (const T*)w.Jp, w.M, w.dpart[2], nullptr, st);
    double v[3];
    pget_status e = host_sums(w, {w.dpart[0], w.dpart[1], w.dpart[2]}, v, st);
    if (e != PGET_OK) return e;
    *pred = -v[0] - 0.5 * v[2] - 0.5 * v[1];
    return PGET_OK;
}

// Shared start of the trial and the check: y and u into the workspace, f(u), prior
// weights and the gradient g = J^T r + alpha grad^T W grad u at u.
template <typename T>
static pget_status at_point(Workspace& w, const pget_lm_params& p, const void* y, const void* lam, const void* mu,
                            double* f, cudaStream_t st) {
    const size_t nn = w.nn, e = w.elt;
    CK(cudaMemcpyAsync(w.yb, y, e * w.M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(w.u, lam, e * nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)w.u + e * nn, mu, e * nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    pack_vec<T>(w, w.u, w.pk_u, nullptr, st);
    pget_status s = objective_at<T>(w, p, w.pk_u, w.u, w.U, w.r, f, st);
    if (s != PGET_OK) return s;
    const T* u = (const T*)w.u;
    reg_weights<T>(u, w.g.n, p.tv_eps, (T*)w.Wl, nullptr, st);
    reg_weights<T>(u + nn, w.g.n, p.tv_eps, (T*)w.Wm, nullptr, st);
    RedArgs<T> ga;
    ga.out = (T*)w.gr;
    ga.v = u;
    ga.Wl = (const T*)w.Wl;
    ga.Wm = (const T*)w.Wm;
    ga.alpha_l = p.alpha_lambda;
    ga.alpha_m = p.alpha_mu;
    set_geo(ga, p, true);
    ga.nu = 0.0;
    CK(op_vjp<T>(w, w.pk_u, w.U, w.r, ga, nullptr, st));
    return PGET_OK;
}

// One trust-region trial at u with damping nu (Alg. 2: s_k = LMA(u_k)); u is not moved.
template <typename T>
static pget_status trial_impl(Workspace& w, const pget_lm_params& p, const void* y, const void* lam,
                              const void* mu, double nu, void* s_out, pget_trial_report* rep, cudaStream_t st) {
    const size_t nn = w.nn;
    memset(rep, 0, sizeof *rep);
    double f = 0.0;
    pget_status s = at_point<T>(w, p, y, lam, mu, &f, st);
    if (s != PGET_OK) return s;
    if (!(nu > 0.0)) {  // nu_0 = nu0_scale |J g|^2 / |g|^2, as at the start of a solve
        dot<T>((const T*)w.gr, (const T*)w.gr, 2 * nn, w.dpart[0], nullptr, st);
        pack_vec<T>(w, w.gr, w.pk_p, nullptr, st);
        CK(op_jvp(w, w.pk_u, w.pk_p, w.Jp, nullptr, st));
        dot<T>((const T*)w.Jp, (const T*)w.Jp, w.M, w.dpart[1], nullptr, st);
        double v[2];
        s = host_sums(w, {w.dpart[0], w.dpart[1]}, v, st);
        if (s != PGET_OK) return s;
        nu = v[0] > 0.0 ? p.nu0_scale * v[1] / v[0] : 1.0;
        if (!(nu > 0.0)) nu = 1.0;
        rep->nu0 = nu;
    }
    s = p.inner_solver == 1 ? run_sgp<T>(w, w.gr, nu, nullptr, p, st) : run_cg<T>(w, w.gr, -1.0, nu, nullptr, p, st);
    if (s != PGET_OK) return s;
    lm_step<T>((const T*)w.u, (const T*)w.x, (T*)w.ut, (T*)w.s, nn, feas_of(p), st);
    double pred = 0.0, ft = 0.0;
    s = model_decrease<T>(w, p, w.s, &pred, st);
    if (s != PGET_OK) return s;
    pack_vec<T>(w, w.ut, w.pk_ut, nullptr, st);
    s = objective_at<T>(w, p, w.pk_ut, w.ut, w.Ut, w.rt, &ft, st);
    if (s != PGET_OK) return s;
    CgState cg;
    CK(cudaMemcpyAsync(&cg, &w.lm->cg, sizeof cg, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s_out, w.s, w.elt * 2 * nn, cudaMemcpyDeviceToDevice, st));
    s = check_err(w, st);
    if (s != PGET_OK) return s;
    const double ared = f - ft;
    const double rho = (pred > 0.0 && std::isfinite(ft)) ? ared / pred : -INFINITY;
    rep->f = f;
    rep->pred = pred;
    rep->ared = ared;
    rep->rho = rho;
    rep->accept = rho > p.eta;
    rep->nu_next = rho < p.rho_lo ? nu * p.nu_up : (rho > p.rho_hi ? nu * p.nu_down : nu);
    rep->cg_iters = cg.iters;
    return PGET_OK;
}

// The safeguard of Prop. conv_check / Alg. 2 for the proposal (pl, pm) at u with the LM
// step s_step: s~ = P(u~) - u (P: projection onto the constraint set); accept iff
// rho(s~) > eta and m_k(s~) <= m_k(s_k).
template <typename T>
static pget_status check_impl(Workspace& w, const pget_lm_params& p, const void* y, const void* lam,
                              const void* mu, const void* s_step, const void* pl, const void* pm,
                              pget_check_report* rep, cudaStream_t st) {
    const size_t nn = w.nn, e = w.elt;
    memset(rep, 0, sizeof *rep);
    double f = 0.0, pred_s = 0.0, pred_p = 0.0, fp = 0.0;
    pget_status s = at_point<T>(w, p, y, lam, mu, &f, st);
    if (s != PGET_OK) return s;
    CK(cudaMemcpyAsync(w.s, s_step, e * 2 * nn, cudaMemcpyDeviceToDevice, st));
    s = model_decrease<T>(w, p, w.s, &pred_s, st);
    if (s != PGET_OK) return s;
    CK(cudaMemcpyAsync(w.ut, pl, e * nn, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)w.ut + e * nn, pm, e * nn, cudaMemcpyDeviceToDevice, st));
    project_set<T>((T*)w.ut, nn, feas_of(p), st);
    sub_dot<T>((const T*)w.ut, (const T*)w.u, (T*)w.s, 2 * nn, w.dpart[3], nullptr, st);
    s = model_decrease<T>(w, p, w.s, &pred_p, st);
    if (s != PGET_OK) return s;
    pack_vec<T>(w, w.ut, w.pk_ut, nullptr, st);
    s = objective_at<T>(w, p, w.pk_ut, w.ut, w.Ut, w.rt, &fp, st);
    if (s != PGET_OK) return s;
    s = check_err(w, st);
    if (s != PGET_OK) return s;
    const double ared = f - fp;
    const double rho = (pred_p > 0.0 && std::isfinite(fp)) ? ared / pred_p : -INFINITY;
    rep->f = f;
    rep->pred_step = pred_s;
    rep->pred_prop = pred_p;
    rep->ared_prop = ared;
    rep->rho_prop = rho;
    rep->accept = rho > p.eta && pred_p >= pred_s;
    return PGET_OK;
}

// Alg. 2 after the trial of iteration k: the proposal's check, then the next iterate in
// (lam, mu): P(u~), else P(u_k + s_k) when the trial was accepted, else u_k.
template <typename T>
static pget_status step_impl(Workspace& w, const pget_lm_params& p0, int k, const void* y, void* lam, void* mu,
                             const void* s_step, const pget_trial_report& tr, double nu0, const void* pl,
                             const void* pm, pget_step_report* rep, cudaStream_t st) {
    const size_t nn = w.nn, e = w.elt;
    const pget_lm_params p = params_at(p0, k);
    memset(rep, 0, sizeof *rep);
    rep->took = tr.accept ? 1 : 0;
    if (pl) {
        pget_status s = check_impl<T>(w, p, y, lam, mu, s_step, pl, pm, &rep->check, st);
        if (s != PGET_OK) return s;
        rep->checked = 1;
        if (rep->check.accept) {  // check_impl left the projected proposal in w.ut
            CK(cudaMemcpyAsync(lam, w.ut, e * nn, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(mu, (const char*)w.ut + e * nn, e * nn, cudaMemcpyDeviceToDevice, st));
            rep->took = 2;
        }
    }
    if (rep->took == 1) {  // u_k + s_k, projected like every iterate
        CK(cudaMemcpyAsync(w.u, lam, e * nn, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync((char*)w.u + e * nn, mu, e * nn, cudaMemcpyDeviceToDevice, st));
        lm_step<T>((const T*)w.u, (const T*)s_step, (T*)w.ut, (T*)w.s, nn, feas_of(p), st);
        CK(cudaMemcpyAsync(lam, w.ut, e * nn, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(mu, (const char*)w.ut + e * nn, e * nn, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    rep->nu_next = std::min(std::max(tr.nu_next, p.nu_min * nu0), p.nu_max * nu0);
    return PGET_OK;
}

template <typename T>
static pget_status init_impl(Workspace& w, const pget_lm_params& p, double mu_init, const void* y, void* lam,
                             void* mu, cudaStream_t st) {
    const size_t nn = w.nn;
    T* u = (T*)w.ut;
    fill<T>(u, nn, 1.0, st);
    const double mu0 = std::min(std::max(mu_init, 0.0), p.mu_max);
    fill<T>(u + nn, nn, mu0, st);
    pack_vec<T>(w, u, w.pk_ut, nullptr, st);
    CK(op_forward(w, w.pk_ut, nullptr, w.Jp, nullptr, st));
    // sum A(1, mu0) and sum y: dot against a vector of ones kept in r
    fill<T>((T*)w.rt, w.M, 1.0, st);
    dot<T>((const T*)w.Jp, (const T*)w.rt, w.M, w.dpart[0], nullptr, st);
    dot<T>((const T*)y, (const T*)w.rt, w.M, w.dpart[1], nullptr, st);
    std::vector<double> a(kRedBlocks), b(kRedBlocks);
    CK(cudaMemcpyAsync(a.data(), w.dpart[0], sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(b.data(), w.dpart[1], sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double sa = 0, sy = 0;
    for (int k = 0; k < kRedBlocks; ++k) {
        sa += a[k];
        sy += b[k];
    }
    double c = sa > 0 ? sy / sa : 0.0;
    c = std::min(std::max(c, 0.0), p.lambda_max);
    fill<T>((T*)lam, nn, c, st);
    fill<T>((T*)mu, nn, mu0, st);
    CK(cudaGetLastError());
    return PGET_OK;
}

}  // namespace

extern "C" {

const char* pget_version(void) { return "pget-gb300 0.1 (sm_103a)"; }

long long pget_launch_count(void) { return pget::launch_count(); }

pget_status pget_profile_enable(pget_ctx* ctx, int32_t enable) {
    return guarded([&]() -> pget_status {
        if (!ctx) return fail(PGET_EINVAL, "null ctx");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        ctx->prof.reset();
        ctx->prof.on = enable != 0;
        return PGET_OK;
    });
}

int32_t pget_profile_read(pget_ctx* ctx, pget_kernel_stat* out, int32_t max) {
    if (!ctx || !out) return 0;
    try {
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        ctx->prof.collect();
        int k = 0;
        for (; k < kPKinds && k < max; ++k) {
            memset(&out[k], 0, sizeof out[k]);
            strncpy(out[k].name, kProfNames[k], sizeof out[k].name - 1);
            out[k].launches = ctx->prof.count[k];
            out[k].total_ms = ctx->prof.total_ms[k];
        }
        return k;
    } catch (...) {  // nothing read: a host-side failure is reported as no entries
        fail(PGET_EINTERNAL, "profile read failed");
        return 0;
    }
}

const char* pget_last_error(pget_ctx*) { return g_last_error.c_str(); }

void pget_default_params(pget_lm_params* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->alpha_lambda = 1e-2;
    o->alpha_mu = 1e-2;
    o->tv_eps = 1e-3;
    o->lambda_max = 2.0;
    o->mu_max = 0.2;
    o->max_iters = 20;
    o->cg_max_iters = 30;
    o->cg_rel_tol = 1e-6;
    o->nu0_scale = 1e-3;
    o->nu_up = 4.0;
    o->nu_down = 0.5;
    o->eta = 1e-3;
    o->rho_lo = 0.25;
    o->rho_hi = 0.75;
    o->nu_min = 1e-12;
    o->nu_max = 1e12;
    o->precision = PGET_F32_KAHAN;
    o->alpha_decay = 1.0;
    o->alpha_decay_iters = 0;
    o->geo_alpha_lambda = 0.0;
    o->geo_alpha_mu = 0.0;
    o->geo_mu_water = 0.0;
    o->geo_mask = nullptr;
    o->inner_solver = 0;
    o->lin_constraint = 0;
    o->lin_slope = 0.0;
    o->lin_offset = 0.0;
}

pget_status pget_create(pget_ctx** ctx, int device, size_t budget) {
    return guarded([&]() -> pget_status {
        if (!ctx) return fail(PGET_EINVAL, "null ctx pointer");
        *ctx = nullptr;
        int nd = 0;
        cudaError_t e = cudaGetDeviceCount(&nd);
        if (e != cudaSuccess) return fail(PGET_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
        if (device < 0 || device >= nd) return fail(PGET_EINVAL, "device %d out of range (%d devices)", device, nd);
        auto c = new (std::nothrow) pget_ctx;
        if (!c) return fail(PGET_ENOMEM, "host allocation failed");
        c->device = device;
        c->budget = budget;
        *ctx = c;
        g_last_error.clear();
        return PGET_OK;
    });
}

pget_status pget_destroy(pget_ctx* ctx) {
    return guarded([&]() -> pget_status {
        if (!ctx) return PGET_OK;
        {
            DeviceGuard dg(ctx->device);
            cudaDeviceSynchronize();
            ctx->slots.clear();
            ctx->pool.clear();
            ctx->batch.reset();
            ctx->ws.reset();
            if (ctx->scratch) cudaFree(ctx->scratch);
        }
        delete ctx;
        return PGET_OK;
    });
}

pget_status pget_forward(pget_ctx* ctx, const pget_geometry* g, int32_t prec, const void* lam, const void* mu,
                         void* y, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_forward");
        if (!ctx || !lam || !mu || !y) return fail(PGET_EINVAL, "null argument");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        pget_status s = get_workspace(ctx, g, prec, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        if (w->f64) pack_pair<double>(*w, lam, mu, w->pk_u, st);
        else pack_pair<float>(*w, lam, mu, w->pk_u, st);
        CK(op_forward(*w, w->pk_u, nullptr, y, nullptr, st));
        return PGET_OK;
    });
}

pget_status pget_jvp(pget_ctx* ctx, const pget_geometry* g, int32_t prec, const void* lam, const void* mu,
                     const void* dlam, const void* dmu, void* dy, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_jvp");
        if (!ctx || !lam || !mu || !dlam || !dmu || !dy) return fail(PGET_EINVAL, "null argument");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        pget_status s = get_workspace(ctx, g, prec, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        if (w->f64) {
            pack_pair<double>(*w, lam, mu, w->pk_u, st);
            pack_pair<double>(*w, dlam, dmu, w->pk_p, st);
        } else {
            pack_pair<float>(*w, lam, mu, w->pk_u, st);
            pack_pair<float>(*w, dlam, dmu, w->pk_p, st);
        }
        CK(op_jvp(*w, w->pk_u, w->pk_p, dy, nullptr, st));
        return PGET_OK;
    });
}


pget_status pget_vjp(pget_ctx* ctx, const pget_geometry* g, int32_t prec, const void* lam, const void* mu,
                     const void* r, void* glam, void* gmu, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_vjp");
        if (!ctx || !lam || !mu || !r || !glam || !gmu) return fail(PGET_EINVAL, "null argument");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        pget_status s = get_workspace(ctx, g, prec, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? vjp_impl<double>(*w, lam, mu, r, glam, gmu, st) : vjp_impl<float>(*w, lam, mu, r, glam, gmu, st);
    });
}

// the batched operators: one workspace, chunks of items per walk launch
static pget_status batch_call(pget_ctx* ctx, const pget_geometry* g, int32_t prec, int32_t batch, int mode,
                              const void* lam, const void* mu, const void* dl, const void* dm, const void* r, void* y,
                              void* gl, void* gm, void* stream) {
    if (!ctx || !lam || !mu) return fail(PGET_EINVAL, "null argument");
    if (batch < 0) return fail(PGET_EINVAL, "batch must be >= 0");
    if (prec == PGET_MIXED) return fail(PGET_EINVAL, "batched operators take PGET_F64, PGET_F32 or PGET_F32_KAHAN");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    Workspace* w;
    pget_status s = get_workspace(ctx, g, prec, &w);
    if (s != PGET_OK || batch == 0) return s;
    cudaStream_t st = (cudaStream_t)stream;
    return w->f64 ? batch_impl<double>(ctx, *w, mode, batch, lam, mu, dl, dm, r, y, gl, gm, st)
                  : batch_impl<float>(ctx, *w, mode, batch, lam, mu, dl, dm, r, y, gl, gm, st);
}

pget_status pget_forward_batch(pget_ctx* ctx, const pget_geometry* g, int32_t prec, int32_t batch, const void* lam,
                               const void* mu, void* y, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_forward_batch");
        if (!y) return fail(PGET_EINVAL, "null argument");
        return batch_call(ctx, g, prec, batch, kFwd, lam, mu, nullptr, nullptr, nullptr, y, nullptr, nullptr, stream);
    });
}

pget_status pget_jvp_batch(pget_ctx* ctx, const pget_geometry* g, int32_t prec, int32_t batch, const void* lam,
                           const void* mu, const void* dlam, const void* dmu, void* dy, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_jvp_batch");
        if (!dlam || !dmu || !dy) return fail(PGET_EINVAL, "null argument");
        return batch_call(ctx, g, prec, batch, kJvp, lam, mu, dlam, dmu, nullptr, dy, nullptr, nullptr, stream);
    });
}

pget_status pget_vjp_batch(pget_ctx* ctx, const pget_geometry* g, int32_t prec, int32_t batch, const void* lam,
                           const void* mu, const void* r, void* glam, void* gmu, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_vjp_batch");
        if (!r || !glam || !gmu) return fail(PGET_EINVAL, "null argument");
        return batch_call(ctx, g, prec, batch, kVjp, lam, mu, nullptr, nullptr, r, nullptr, glam, gmu, stream);
    });
}

pget_status pget_operator_status(pget_ctx* ctx, void* stream) {
    return guarded([&]() -> pget_status {
        if (!ctx) return fail(PGET_EINVAL, "null ctx");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        if (!ctx->ws) return PGET_OK;  // no operator call yet
        cudaStream_t st = (cudaStream_t)stream;
        Workspace& w = *ctx->ws;
        CK(cudaMemcpyAsync(w.host_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
        CK(cudaStreamSynchronize(st));
        return flags_status(*w.host_err);
    });
}

pget_status pget_reg_apply(pget_ctx* ctx, int32_t n, int32_t prec, double alpha, double eps, const void* u,
                           const void* v, void* out, double* value_host, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_reg_apply");
        if (!ctx || !u || !v || !out) return fail(PGET_EINVAL, "null argument");
        if (n < 2) return fail(PGET_EINVAL, "n must be >= 2");
        if (!known_precision(prec)) return fail(PGET_EINVAL, "unknown precision");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        cudaStream_t st = (cudaStream_t)stream;
        const size_t elt = vectors_f64(prec) ? 8 : 4;
        const size_t need = elt * (size_t)n * n + sizeof(double) * (kRedBlocks + 1);
        if (ctx->scratch_bytes < need) {
            CK(cudaStreamSynchronize(st));
            if (ctx->scratch) cudaFree(ctx->scratch);
            ctx->scratch = nullptr;
            ctx->scratch_bytes = 0;
            CK(cudaMalloc(&ctx->scratch, need));
            ctx->scratch_bytes = need;
        }
        double* part = (double*)ctx->scratch;
        void* W = (char*)ctx->scratch + sizeof(double) * (kRedBlocks + 1);
        if (vectors_f64(prec)) {
            reg_weights<double>((const double*)u, n, eps, (double*)W, nullptr, st);
            reg_apply<double>((const double*)v, (const double*)W, n, alpha, (double*)out, st);
            if (value_host) reg_value<double>((const double*)u, n, alpha, eps, part, nullptr, st);
        } else {
            reg_weights<float>((const float*)u, n, eps, (float*)W, nullptr, st);
            reg_apply<float>((const float*)v, (const float*)W, n, alpha, (float*)out, st);
            if (value_host) reg_value<float>((const float*)u, n, alpha, eps, part, nullptr, st);
        }
        CK(cudaGetLastError());
        if (value_host) {
            finish_sum(part, part + kRedBlocks, nullptr, st);
            CK(cudaMemcpyAsync(value_host, part + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        return PGET_OK;
    });
}


pget_status pget_cg_solve(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* lam,
                          const void* mu, double nu, const void* rhs, void* x, int32_t* iters, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_cg_solve");
        if (!ctx || !lam || !mu || !rhs || !x) return fail(PGET_EINVAL, "null argument");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        if (!(nu >= 0) || !std::isfinite(nu)) return fail(PGET_EINVAL, "nu must be finite and >= 0");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? cg_impl<double>(*w, *p, lam, mu, nu, rhs, x, iters, st)
                      : cg_impl<float>(*w, *p, lam, mu, nu, rhs, x, iters, st);
    });
}


pget_status pget_initial_guess(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, double mu_init,
                               const void* y, void* lam, void* mu, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_initial_guess");
        if (!ctx || !y || !lam || !mu) return fail(PGET_EINVAL, "null argument");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? init_impl<double>(*w, *p, mu_init, y, lam, mu, st)
                      : init_impl<float>(*w, *p, mu_init, y, lam, mu, st);
    });
}

pget_status pget_lm_trial(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* y,
                          const void* lam, const void* mu, double nu, void* s_out, pget_trial_report* rep,
                          void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_lm_trial");
        if (!ctx || !y || !lam || !mu || !s_out || !rep) return fail(PGET_EINVAL, "null argument");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? trial_impl<double>(*w, *p, y, lam, mu, nu, s_out, rep, st)
                      : trial_impl<float>(*w, *p, y, lam, mu, nu, s_out, rep, st);
    });
}

pget_status pget_proposal_check(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* y,
                                const void* lam, const void* mu, const void* s_step, const void* prop_lam,
                                const void* prop_mu, pget_check_report* rep, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_proposal_check");
        if (!ctx || !y || !lam || !mu || !s_step || !prop_lam || !prop_mu || !rep)
            return fail(PGET_EINVAL, "null argument");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? check_impl<double>(*w, *p, y, lam, mu, s_step, prop_lam, prop_mu, rep, st)
                      : check_impl<float>(*w, *p, y, lam, mu, s_step, prop_lam, prop_mu, rep, st);
    });
}

pget_status pget_lm_step_with_proposal(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, int32_t k,
                                       const void* y, void* lam, void* mu, const void* s_step,
                                       const pget_trial_report* trial, double nu0, const void* pl, const void* pm,
                                       pget_step_report* rep, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_lm_step_with_proposal");
        if (!ctx || !y || !lam || !mu || !s_step || !trial || !rep) return fail(PGET_EINVAL, "null argument");
        if ((pl == nullptr) != (pm == nullptr)) return fail(PGET_EINVAL, "give both proposal images or neither");
        if (k < 0) return fail(PGET_EINVAL, "iteration k must be >= 0");
        if (!(nu0 > 0.0) || !std::isfinite(nu0)) return fail(PGET_EINVAL, "nu0 must be finite and > 0");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? step_impl<double>(*w, *p, k, y, lam, mu, s_step, *trial, nu0, pl, pm, rep, st)
                      : step_impl<float>(*w, *p, k, y, lam, mu, s_step, *trial, nu0, pl, pm, rep, st);
    });
}

pget_status pget_params_at(const pget_lm_params* p, int32_t k, pget_lm_params* out) {
    return guarded([&]() -> pget_status {
        if (!p || !out) return fail(PGET_EINVAL, "null argument");
        if (k < 0) return fail(PGET_EINVAL, "iteration k must be >= 0");
        *out = params_at(*p, k);
        return PGET_OK;
    });
}

pget_status pget_check_params(const pget_lm_params* p) {
    return guarded([&]() -> pget_status { return check_params(p); });
}

pget_status pget_geometry_info(const pget_geometry* gin, int32_t* n_samples, int32_t* n_banks, double* fov_radius,
                               double* det_pitch, int32_t* max_slots) {
    return guarded([&]() -> pget_status {
        if (!gin) return fail(PGET_EINVAL, "null geometry");
        Geometry g;
        std::string msg;
        pget_status s = build_geometry(*gin, &g, &msg);
        if (s != PGET_OK) return fail(s, "%s", msg.c_str());
        if (n_samples) *n_samples = g.T;
        if (n_banks) *n_banks = g.n_banks;
        if (fov_radius) *fov_radius = g.r;
        if (det_pitch) *det_pitch = g.p;
        if (max_slots) *max_slots = g.max_slots;
        return PGET_OK;
    });
}

pget_status pget_walk_plans(const pget_geometry* gin, int32_t precision, pget_walk_plan_info* out) {
    return guarded([&]() -> pget_status {
        if (!gin || !out) return fail(PGET_EINVAL, "null argument");
        if (!known_precision(precision)) return fail(PGET_EINVAL, "unknown precision %d", precision);
        Geometry g;
        std::string msg;
        pget_status s = build_geometry(*gin, &g, &msg);
        if (s != PGET_OK) return fail(s, "%s", msg.c_str());
        WalkPlan pl[3];
        walk_plans(g, ((g.n + 2 + 1) / 2) * 2, walk_precision(precision) == PGET_F64, &pl[0], &pl[1], &pl[2]);
        out->threads = pl[0].threads;
        for (int k = 0; k < 3; ++k) {
            out->rows_per_chunk[k] = pl[k].Yc;
            out->chunks[k] = pl[k].nchunks;
            out->smem_bytes[k] = (int32_t)pl[k].smem;
        }
        out->adjoint_phases = pl[2].nph;
        out->phases_needed = adjoint_phases_needed(g);
        return PGET_OK;
    });
}

pget_status pget_project(pget_ctx* ctx, const pget_lm_params* p, int32_t n, void* lam, void* mu, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_project");
        if (!ctx || !lam || !mu) return fail(PGET_EINVAL, "null argument");
        if (n < 1) return fail(PGET_EINVAL, "n must be >= 1");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        cudaStream_t st = (cudaStream_t)stream;
        const size_t nn = (size_t)n * n;
        if (vectors_f64(p->precision)) project_pair<double>((double*)lam, (double*)mu, nn, feas_of(*p), st);
        else project_pair<float>((float*)lam, (float*)mu, nn, feas_of(*p), st);
        CK(cudaGetLastError());
        return PGET_OK;
    });
}

pget_status pget_lm_solve(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* y,
                          void* lam_io, void* mu_io, pget_lm_report* rep, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_lm_solve");
        if (!ctx || !y || !lam_io || !mu_io) return fail(PGET_EINVAL, "null argument");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        return w->f64 ? lm_solve_impl<double>(*w, *p, y, lam_io, mu_io, lam_io, mu_io, rep, st)
                      : lm_solve_impl<float>(*w, *p, y, lam_io, mu_io, lam_io, mu_io, rep, st);
    });
}

pget_status pget_lm_solve_host(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* y_host,
                               void* lam_host, void* mu_host, int32_t init_guess, pget_lm_report* rep, void* stream) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_lm_solve_host");
        if (!ctx || !y_host || !lam_host || !mu_host) return fail(PGET_EINVAL, "null argument");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Workspace* w;
        s = get_workspace(ctx, g, p->precision, &w);
        if (s != PGET_OK) return s;
        cudaStream_t st = (cudaStream_t)stream;
        const size_t nn = w->nn, e = w->elt;
        // inputs: y into the measured-data buffer, the initial guess into x (the solve copies
        // it into the iterate before CG first writes x)
        CK(cudaMemcpyAsync(w->yb, y_host, e * w->M, cudaMemcpyHostToDevice, st));
        void* ld = w->x;
        void* md = (char*)w->x + e * nn;
        if (init_guess) {
            s = w->f64 ? init_impl<double>(*w, *p, 0.01, w->yb, ld, md, st)
                       : init_impl<float>(*w, *p, 0.01, w->yb, ld, md, st);
            if (s != PGET_OK) return s;
        } else {
            CK(cudaMemcpyAsync(ld, lam_host, e * nn, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(md, mu_host, e * nn, cudaMemcpyHostToDevice, st));
        }
        void* lx = w->x;
        void* mx = (char*)w->x + e * nn;
        s = w->f64 ? lm_solve_impl<double>(*w, *p, w->yb, lx, mx, w->q, (char*)w->q + e * nn, rep, st)
                   : lm_solve_impl<float>(*w, *p, w->yb, lx, mx, w->q, (char*)w->q + e * nn, rep, st);
        if (s != PGET_OK) return s;
        CK(cudaMemcpyAsync(lam_host, w->q, e * nn, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(mu_host, (char*)w->q + e * nn, e * nn, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return PGET_OK;
    });
}

pget_status pget_submit(pget_ctx* ctx, const pget_geometry* g, const pget_lm_params* p, const void* y,
                        const void* lam0, const void* mu0, uint64_t* ticket) {
    return guarded([&]() -> pget_status {
        PGET_RANGE("pget_submit");
        if (!ctx || !y || !ticket) return fail(PGET_EINVAL, "null argument");
        if ((lam0 == nullptr) != (mu0 == nullptr)) return fail(PGET_EINVAL, "give both lam0 and mu0, or neither");
        pget_status s = check_params(p);
        if (s != PGET_OK) return s;
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        Geometry geo;
        std::string key;
        int groups = 1;
        size_t need = 0;
        s = resolve(g, p->precision, &geo, &key, &groups, &need);
        if (s != PGET_OK) return s;
        if (ctx->budget && need > ctx->budget)
            return fail(PGET_ENOMEM, "request needs %zu bytes of workspace, budget is %zu", need, ctx->budget);
        if (ctx->slots.empty())
            for (int k = 0; k < max_inflight(); ++k) ctx->slots.emplace_back(new Slot);
        // a free slot, preferably one whose cached workspace fits this request as is
        Slot* sl = nullptr;
        for (auto& c : ctx->slots)
            if (c->state == Slot::kFree && c->ws && c->ws_key == key) {
                sl = c.get();
                break;
            }
        if (!sl)
            for (auto& c : ctx->slots)
                if (c->state == Slot::kFree && !c->ws) {
                    sl = c.get();
                    break;
                }
        if (!sl)
            for (auto& c : ctx->slots)
                if (c->state == Slot::kFree) {
                    sl = c.get();
                    break;
                }
        if (!sl) return fail(PGET_EAGAIN, "all %zu serving slots are busy", ctx->slots.size());
        if (!(sl->ws && sl->ws_key == key)) {
            // park the slot's workspace (idle: its last request was collected) and take an
            // idle one of this geometry if there is one
            if (sl->ws) ctx->pool.push_back({sl->ws_key, std::move(sl->ws), ++ctx->use_clock});
            sl->ws_key.clear();
            for (size_t i = 0; i < ctx->pool.size(); ++i)
                if (ctx->pool[i].key == key) {
                    sl->ws = std::move(ctx->pool[i].ws);
                    sl->ws_key = key;
                    ctx->pool.erase(ctx->pool.begin() + i);
                    break;
                }
        }
        if (!sl->ws) {
            // a new workspace: make room by freeing idle ones, least recently used first
            auto held = [&] { return serving_bytes(ctx) + (ctx->ws ? ctx->ws->bytes : 0); };
            const size_t cap = ctx->budget ? ctx->budget : default_serving_cap();
            while (held() + need > cap && evict_idle(ctx)) {
            }
            if (ctx->budget && held() + need > ctx->budget)
                return fail(PGET_EAGAIN, "device memory budget in use (%zu of %zu bytes held, %zu needed)", held(),
                            ctx->budget, need);
            std::unique_ptr<Workspace> w;
            s = make_workspace(ctx, std::move(geo), p->precision, groups, &w);
            if (s != PGET_OK) return s;
            sl->ws = std::move(w);
            sl->ws_key = key;
        }
        if (!sl->stream) CK(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
        if (!sl->done) CK(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
        Workspace& w = *sl->ws;
        cudaStream_t st = sl->stream;
        const size_t nn = w.nn, e = w.elt;
        // inputs into slot memory; the caller may free its buffers when this call returns
        CK(cudaMemcpyAsync(w.yb, y, e * w.M, cudaMemcpyDeviceToDevice, st));
        if (lam0) {
            CK(cudaMemcpyAsync(w.u, lam0, e * nn, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync((char*)w.u + e * nn, mu0, e * nn, cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaStreamSynchronize(st));
        if (!lam0) {
            s = w.f64 ? init_async<double>(w, *p, 0.01, w.u, (char*)w.u + e * nn, st)
                      : init_async<float>(w, *p, 0.01, w.u, (char*)w.u + e * nn, st);
            if (s != PGET_OK) return s;
        }
        s = w.f64 ? lm_launch<double>(w, *p, st) : lm_launch<float>(w, *p, st);
        if (s != PGET_OK) return s;
        CK(cudaEventRecord(sl->done, st));
        sl->state = Slot::kRunning;
        sl->ticket = ctx->next_ticket++;
        *ticket = sl->ticket;
        return PGET_OK;
    });
}

pget_status pget_poll(pget_ctx* ctx, uint64_t ticket, void* lam_out, void* mu_out, pget_lm_report* rep, int* done) {
    return guarded([&]() -> pget_status {
        if (!ctx || !done) return fail(PGET_EINVAL, "null argument");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        *done = 0;
        Slot* sl = nullptr;
        for (auto& c : ctx->slots)
            if (c->state != Slot::kFree && c->ticket == ticket) sl = c.get();
        if (!sl) return fail(PGET_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        if (sl->state == Slot::kRunning) {
            cudaError_t q = cudaEventQuery(sl->done);
            if (q == cudaErrorNotReady) return PGET_OK;
            if (q != cudaSuccess) {
                sl->state = Slot::kFree;
                sl->ws.reset();
                sl->ws_key.clear();
                *done = 1;
                return fail(PGET_ECUDA, "request %llu: %s", (unsigned long long)ticket, cudaGetErrorString(q));
            }
            sl->state = Slot::kDone;
        }
        Workspace& w = *sl->ws;
        const size_t nn = w.nn, e = w.elt;
        if (lam_out) CK(cudaMemcpyAsync(lam_out, w.u, e * nn, cudaMemcpyDeviceToDevice, sl->stream));
        if (mu_out) CK(cudaMemcpyAsync(mu_out, (char*)w.u + e * nn, e * nn, cudaMemcpyDeviceToDevice, sl->stream));
        CK(cudaStreamSynchronize(sl->stream));
        pget_status s = lm_finish(w, rep);
        sl->state = Slot::kFree;
        *done = 1;
        return s;
    });
}

pget_status pget_cancel(pget_ctx* ctx, uint64_t ticket) {
    return guarded([&]() -> pget_status {
        if (!ctx) return fail(PGET_EINVAL, "null ctx");
        std::lock_guard<std::mutex> lk(ctx->mu);
        DeviceGuard dg(ctx->device);
        for (auto& c : ctx->slots)
            if (c->state != Slot::kFree && c->ticket == ticket) {
                // kernels cannot be aborted once queued: wait for them, then drop the result
                cudaStreamSynchronize(c->stream);
                c->state = Slot::kFree;
                return PGET_OK;
            }
        return fail(PGET_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    });
}

int32_t pget_inflight(pget_ctx* ctx) {
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    int k = 0;
    for (auto& c : ctx->slots) k += c->state != Slot::kFree;
    return k;
}

}  // extern "C"
