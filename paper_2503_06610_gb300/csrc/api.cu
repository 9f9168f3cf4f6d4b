// api.cu -- the C ABI of include/nh.h: contexts, workspace layout, the hybrid
// scheduler of arXiv:2503.06610 Sec. II.D (one fused LB launch per step; every
// dt_FD steps the FD predictor, corrector, stress and force launches), CUDA
// graphs for whole dt_FD blocks, per-kernel timing and diagnostics.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "nh_internal.cuh"

#include <cstddef>

#include <nvtx3/nvToolsExt.h>

using namespace nh;

// The parameter block is passed by pointer from C and from Python's ctypes:
// 16 int32 fields then 18 doubles, without padding.
static_assert(sizeof(nh_params) == 16 * 4 + 18 * 8, "nh_params layout");
static_assert(offsetof(nh_params, tau) == 64, "nh_params layout");

namespace {

thread_local std::string g_global_err;

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t real_size(const nh_params& p) { return p.precision == NH_FP64 ? 8 : 4; }
size_t store_size(const nh_params& p)
{
    switch (p.storage) {
    case NH_STORE_F64: return 8;
    case NH_STORE_F32: return 4;
    default: return 2;
    }
}

struct Layout {
    size_t f[2], F, Fprev, n, nP, ndot, u, rho, sigma, P3, snap, staging, partials, result, scales, absmax, trig, solid,
        lbpart, bpart, tubesd, total;
};

Layout make_layout(const nh_params& p)
{
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    const size_t R = real_size(p), S = store_size(p);
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    L.f[0] = take(19 * N * S);
    L.f[1] = take(19 * N * S);
    L.F = take(3 * N * R);
    L.Fprev = take(p.paper_order ? 3 * N * R : 0);  // the force of the previous FD interval
    L.n = take(3 * N * R);
    L.nP = take(3 * N * R);
    L.ndot = take(3 * N * R);
    L.u = take(3 * N * R);
    L.rho = take(N * R);
    L.sigma = take(9 * N * R);
    L.P3 = take(p.frank3 ? 9 * N * R : 0);  // d df/d(grad n) of the three-constant correction
    L.snap = take(3 * N * R);
    L.staging = take(7 * N * sizeof(double));
    L.partials = take((size_t)diag_blocks() * diag_num_values(NH_MAX_TUBES) * sizeof(double));
    L.result = take((size_t)diag_num_values(NH_MAX_TUBES) * sizeof(double));
    L.scales = take(4 * sizeof(float));
    L.absmax = take(4 * sizeof(float));
    L.trig = take(2 * ((size_t)p.nx + p.ny) * sizeof(double));
    L.solid = take(N);  // obstacle mask, 1 byte per site (used after nh_set_solid)
    // diagnostics partials of a macro LB launch: [3][blocks], at most one block per 128 sites
    L.lbpart = take(3 * ((N + 127) / 128 + 1) * sizeof(double));
    // diagnostics partials of the fused stress kernel: [V][blocks], at most one block per 32 x 8 columns and layer
    const size_t fd_tiles = (size_t)((p.nx + 31) / 32) * ((p.ny + 7) / 8) * p.nz;
    L.bpart = take(fd_tiles * diag_num_values(NH_MAX_TUBES) * sizeof(double));
    L.tubesd = take(2 * NH_MAX_TUBES * sizeof(double));  // previous tube centroids on the device
    L.total = off;
    return L;
}

int validate(const nh_params* p, std::string& err)
{
    if (!p) {
        err = "params is NULL";
        return NH_EINVAL;
    }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) {
        err = "nx, ny, nz must be >= 1";
        return NH_EINVAL;
    }
    const double N = (double)p->nx * p->ny * p->nz;
    if (19.0 * N > 2147483647.0) {
        err = "domain too large: 19*nx*ny*nz must fit in a signed 32-bit index";
        return NH_EINVAL;
    }
    if (!(p->tau > 0.5) || !isfinite(p->tau)) {
        err = "tau must be > 1/2";
        return NH_EINVAL;
    }
    if (!(p->gamma1 > 0.0)) {
        err = "gamma1 must be > 0";
        return NH_EINVAL;
    }
    if (p->dt_fd < 1) {
        err = "dt_fd must be >= 1";
        return NH_EINVAL;
    }
    if (p->walls_z != 0 && p->walls_z != 1) {
        err = "walls_z must be 0 or 1";
        return NH_EINVAL;
    }
    if (p->anchoring != NH_ANCHOR_NONE && p->anchoring != NH_ANCHOR_HOMEOTROPIC) {
        err = "anchoring must be NH_ANCHOR_NONE or NH_ANCHOR_HOMEOTROPIC";
        return NH_EINVAL;
    }
    if (p->precision == NH_FP64) {
        if (p->storage != NH_STORE_F64) {
            err = "FP64 precision requires NH_STORE_F64";
            return NH_EINVAL;
        }
    } else if (p->precision == NH_FP32) {
        if (p->storage != NH_STORE_F32 && p->storage != NH_STORE_F16S && p->storage != NH_STORE_BF16S) {
            err = "FP32 precision requires NH_STORE_F32, NH_STORE_F16S or NH_STORE_BF16S";
            return NH_EINVAL;
        }
        if ((p->storage == NH_STORE_F16S || p->storage == NH_STORE_BF16S) && !p->shifted) {
            err = "16-bit population stores hold shifted populations: set shifted = 1";
            return NH_EINVAL;
        }
    } else {
        err = "precision must be NH_FP64 or NH_FP32";
        return NH_EINVAL;
    }
    if (p->shifted != 0 && p->shifted != 1) {
        err = "shifted must be 0 or 1";
        return NH_EINVAL;
    }
    if (p->paper_order != 0 && p->paper_order != 1) {
        err = "paper_order must be 0 or 1";
        return NH_EINVAL;
    }
    if (p->frank3 != 0 && p->frank3 != 1) {
        err = "frank3 must be 0 or 1";
        return NH_EINVAL;
    }
    const int32_t flags[] = {p->renorm_predictor, p->lap_wide, p->n_from_rate, p->ghost_sigma};
    for (int32_t f : flags)
        if (f != 0 && f != 1) {
            err = "renorm_predictor, lap_wide, n_from_rate and ghost_sigma must be 0 or 1";
            return NH_EINVAL;
        }
    if (p->frank3 && !(p->K11 > 0 && p->K22 > 0 && p->K33 > 0 && isfinite(p->K11) && isfinite(p->K22) &&
                       isfinite(p->K33))) {
        err = "frank3 needs finite K11, K22, K33 > 0";
        return NH_EINVAL;
    }
    const double vals[] = {p->g[0], p->g[1], p->g[2], p->K, p->q0, p->gamma2, p->alpha1, p->alpha2,
                           p->alpha3, p->alpha4p, p->alpha5, p->alpha6, p->W0};
    for (double v : vals)
        if (!isfinite(v)) {
            err = "non-finite parameter";
            return NH_EINVAL;
        }
    if (p->check_stability && p->dt_fd * 6.0 * p->K / p->gamma1 > 1.0) {
        err = "dt_fd * 6 K / gamma1 > 1: the predictor-corrector is unstable on the compact Laplacian";
        return NH_EINVAL;
    }
    return NH_OK;
}

}  // namespace

void nh::set_global_error(const char* msg) { g_global_err = msg ? msg : ""; }

int nh::validate_params(const nh_params* p, std::string& err) { return validate(p, err); }

namespace {

// A run of consecutive launches of one kernel class on one stream, bracketed
// by one pair of CUDA events.
struct TimedLaunch {
    int kclass;
    cudaEvent_t a, b;
    int count;
};

}  // namespace

struct nh_ctx {
    nh_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int N = 0;
    Layout L{};
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool bound = false;
    bool fields_set = false;
    bool has_solid = false;  // an obstacle mask is set (nh_set_solid)
    int64_t n_fluid = 0;     // fluid sites when has_solid
    int cur = 0;
    int64_t step = 0;
    std::string err;
    int n_tubes = 0;
    double tubes[NH_MAX_TUBES][2] = {};
    bool use_graphs = true;
    int lb_variant = 0;
    int fd_fused = 1;  // 1: fused 2.5D FD kernels; 0: per-site kernels
    int sm_count = 152;
    int64_t epoch = 0;  // bumped whenever buffers or launch shapes change (invalidates batch plans)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
    int timing = 0;  // 0 off, 1 every kernel class, 2 the LB class only
    std::vector<TimedLaunch> pending;
    bool seg_open = false;
    TimedLaunch seg{};
    cudaStream_t seg_stream = nullptr;
    std::vector<cudaEvent_t> free_events;
    nh_timing tstats{};
    int64_t launches = 0;
    double host_result[6 + 5 * NH_MAX_TUBES] = {};
    bool diag_pending = false;
    bool snap_valid = false;  // a director snapshot exists (nh_director_change)
    int diag_tubes = 0;
    cudaStream_t diag_stream = nullptr;
    double wait_limit = 0.0;  // seconds; > 0 bounds the host-side waits (nh_set_wait_limit)
    int diag_fold = 1;        // macro LB launches leave the diagnostics' population, u and rho sums
    int64_t lbp_step = -1;    // step whose state those sums describe (-1: none)
    int lbp_blocks = 0;       // blocks of the launch that wrote them
    int64_t bdp_step = -1;    // step of the director whose diagnostics partials the fused stress kernel left
    int bdp_blocks = 0;
    int64_t tubes_epoch = 0;  // counts changes of the previous tube centroids (tubes, device copy at L.tubesd)
    int64_t bdp_tubes_epoch = -1;  // the centroids those partials were assigned with
    bool tubes_dirty = true;       // the device copy lags the host centroids

    template <typename T>
    T* at(size_t off) const
    {
        return reinterpret_cast<T*>(ws + off);
    }
};

namespace {

int fail(nh_ctx* c, int code, const std::string& msg)
{
    if (c)
        c->err = msg;
    else
        g_global_err = msg;
    return code;
}

int cuda_fail(nh_ctx* c, cudaError_t e, const char* where)
{
    return fail(c, NH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define NH_CUDA(ctx, ...)                                                   \
    do {                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #__VA_ARGS__);   \
    } while (0)

cudaStream_t pick(nh_ctx* c, void* s) { return s ? static_cast<cudaStream_t>(s) : c->stream; }

// Wait for the work enqueued on st, for at most the context's wait limit:
// NH_ETIMEOUT (work left running) when the limit passes first.  Without a
// limit this returns at once and the caller's own synchronisation waits.
int bounded_wait(nh_ctx* c, cudaStream_t st)
{
    if (!(c->wait_limit > 0.0)) return NH_OK;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return NH_OK;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "cudaStreamQuery");
        const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (waited > c->wait_limit)
            return fail(c, NH_ETIMEOUT,
                        "the stream did not finish within the wait limit of " + std::to_string(c->wait_limit) + " s");
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

// NVTX range around an API call that enqueues GPU work (visible in profilers).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

void drop_batch_plans(const nh_ctx* c);

void drop_graphs(nh_ctx* c)
{
    c->epoch += 1;
    drop_batch_plans(c);
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_kernels[k] = 0;
    }
}

cudaEvent_t get_event(nh_ctx* c)
{
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// ------------------------------------------------------------ launch helpers

template <typename Real, typename Store>
LBChan<Real, Store> lb_chan(nh_ctx* c, int src)
{
    LBChan<Real, Store> a;
    a.fsrc = c->at<const Store>(c->L.f[src]);
    a.fdst = c->at<Store>(c->L.f[1 - src]);
    a.F = c->at<const Real>(c->L.F);
    a.Fu = nullptr;
    a.solid = c->has_solid ? c->at<const unsigned char>(c->L.solid) : nullptr;
    a.u = c->at<Real>(c->L.u);
    a.rho = c->at<Real>(c->L.rho);
    a.scales = c->at<float>(c->L.scales);
    a.ctrl = c->at<unsigned>(c->L.absmax);
    a.part = nullptr;
    a.src = src;
    a.g = Geom{c->p.nx, c->p.ny, c->p.nz, c->p.walls_z, c->p.anchoring, c->N};
    a.omega = Real(1.0 / c->p.tau);
    a.gx = Real(c->p.g[0]);
    a.gy = Real(c->p.g[1]);
    a.gz = Real(c->p.g[2]);
    return a;
}

template <typename Real>
FDChan<Real> fd_chan(nh_ctx* c)
{
    FDChan<Real> a;
    a.n = c->at<Real>(c->L.n);
    a.nP = c->at<Real>(c->L.nP);
    a.ndot = c->at<Real>(c->L.ndot);
    a.u = c->at<const Real>(c->L.u);
    a.sigma = c->at<Real>(c->L.sigma);
    a.F = c->at<Real>(c->L.F);
    a.P3 = c->p.frank3 ? c->at<Real>(c->L.P3) : nullptr;
    a.solid = c->has_solid ? c->at<const unsigned char>(c->L.solid) : nullptr;
    a.g = Geom{c->p.nx, c->p.ny, c->p.nz, c->p.walls_z, c->p.anchoring, c->N};
    const nh_params& p = c->p;
    a.p.K = Real(p.K);
    a.p.q0 = Real(p.q0);
    a.p.W0 = Real(p.W0);
    a.p.inv_gamma1 = Real(1.0 / p.gamma1);
    a.p.gamma2 = Real(p.gamma2);
    a.p.g2_over_g1 = Real(p.gamma2 / p.gamma1);
    a.p.a1 = Real(p.alpha1);
    a.p.a2 = Real(p.alpha2);
    a.p.a3 = Real(p.alpha3);
    a.p.a4p = Real(p.alpha4p);
    a.p.a5 = Real(p.alpha5);
    a.p.a6 = Real(p.alpha6);
    a.p.dt = Real(p.dt_fd);
    a.p.kd1 = Real(p.frank3 ? p.K11 - p.K : 0.0);
    a.p.kd2 = Real(p.frank3 ? p.K22 - p.K : 0.0);
    a.p.kd3 = Real(p.frank3 ? p.K33 - p.K : 0.0);
    const double lam = p.gamma2 / p.gamma1;
    a.p.kg = Real(p.K / p.gamma1);
    a.p.kqg = Real(p.K * p.q0 / p.gamma1);
    a.p.w0g = Real(p.W0 / p.gamma1);
    a.p.c1 = Real(0.25 * (1.0 - lam));
    a.p.c2 = Real(-0.25 * (1.0 + lam));
    a.p.kq = Real(p.K * p.q0);
    a.p.g2q = Real(0.25 * lam);
    a.p.a1q = Real(0.25 * p.alpha1);
    a.p.a4q = Real(0.25 * p.alpha4p);
    a.p.a5q = Real(0.25 * p.alpha5);
    a.p.a6q = Real(0.25 * p.alpha6);
    a.p.k4 = Real(0.25 * p.K);
    a.p.kq2 = Real(0.5 * p.K * p.q0);
    a.p.renorm_p = p.renorm_predictor;
    a.p.lap_wide = p.lap_wide;
    a.p.n_rate = 0;  // set by the caller for the force that follows an FD update
    a.p.mirror = p.ghost_sigma;
    return a;
}

// Close the open timing segment (records its end event).
void close_segment(nh_ctx* c)
{
    if (!c->seg_open) return;
    cudaEventRecord(c->seg.b, c->seg_stream);
    c->pending.push_back(c->seg);
    c->seg_open = false;
}

// Enqueue one kernel launch of class kclass.  With timing on, consecutive
// launches of the same class on the same stream form one segment bracketed by
// a single pair of events (the per-launch time is segment time / count).
template <typename F>
int timed(nh_ctx* c, int kclass, cudaStream_t st, F&& launch, const char* what)
{
    const bool timed_class = c->timing == 1 || (c->timing == 2 && kclass == NH_KCLASS_LB);
    if (c->seg_open && (!timed_class || c->seg.kclass != kclass || c->seg_stream != st)) close_segment(c);
    if (timed_class && !c->seg_open) {
        c->seg = TimedLaunch{kclass, get_event(c), get_event(c), 0};
        c->seg_stream = st;
        cudaEventRecord(c->seg.a, st);
        c->seg_open = true;
    }
    cudaError_t e = launch();
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    if (timed_class) c->seg.count += 1;
    c->launches += 1;
    return NH_OK;
}

// The diagnostics can take the population, u and rho sums from the macro LB
// launch that wrote the state (F32 / F64 stores, no obstacles, and not with
// the printed loop order, whose macro launch's populations are replaced).
bool fold_ok(const nh_ctx* c)
{
    return c->diag_fold && !c->p.paper_order && !c->has_solid &&
           (c->p.storage == NH_STORE_F32 || c->p.storage == NH_STORE_F64);
}

// One LB launch from population buffer src.  stale_u: u is shifted by half of
// the previous FD interval's force (Fprev) instead of the current one.  A
// macro launch (write_macro) also leaves the diagnostics' sums when fold_ok.
int enqueue_lb(nh_ctx* c, int src, bool write_macro, cudaStream_t st, bool stale_u = false)
{
    const bool sh = c->p.shifted != 0;
    const bool fold = write_macro && fold_ok(c);
    if (fold) {
        c->lbp_step = c->step + 1;
        c->lbp_blocks = lb_blocks(c->lb_variant, c->N);
    }
    switch (c->p.storage) {
    case NH_STORE_F64: {
        auto a = lb_chan<double, double>(c, src);
        if (stale_u) a.Fu = c->at<const double>(c->L.Fprev);
        if (fold) a.part = c->at<double>(c->L.lbpart);
        return timed(c, NH_KCLASS_LB, st, [&] { return launch_lb(a, sh, write_macro, c->lb_variant, st); }, "lb");
    }
    case NH_STORE_F32: {
        auto a = lb_chan<float, float>(c, src);
        if (stale_u) a.Fu = c->at<const float>(c->L.Fprev);
        if (fold) a.part = c->at<double>(c->L.lbpart);
        return timed(c, NH_KCLASS_LB, st, [&] { return launch_lb(a, sh, write_macro, c->lb_variant, st); }, "lb");
    }
    case NH_STORE_F16S: {
        auto a = lb_chan<float, __half>(c, src);
        if (stale_u) a.Fu = c->at<const float>(c->L.Fprev);
        return timed(c, NH_KCLASS_LB, st, [&] { return launch_lb(a, sh, write_macro, c->lb_variant, st); }, "lb");
    }
    default: {
        auto a = lb_chan<float, __nv_bfloat16>(c, src);
        if (stale_u) a.Fu = c->at<const float>(c->L.Fprev);
        return timed(c, NH_KCLASS_LB, st, [&] { return launch_lb(a, sh, write_macro, c->lb_variant, st); }, "lb");
    }
    }
}

// Per-site predictor and corrector; with the three-constant energy each is
// preceded by the P stage of the field it differentiates.
template <typename Real>
int enqueue_predict_correct_sites(nh_ctx* c, const FDChan<Real>& a, cudaStream_t st)
{
    int r = NH_OK;
    if (a.P3) r = timed(c, NH_KCLASS_FD_PREDICT, st, [&] { return launch_frank3_p(a, false, st); }, "frank3_p");
    if (r) return r;
    r = timed(c, NH_KCLASS_FD_PREDICT, st, [&] { return launch_fd_predict(a, st); }, "fd_predict");
    if (r) return r;
    if (a.P3) r = timed(c, NH_KCLASS_FD_CORRECT, st, [&] { return launch_frank3_p(a, true, st); }, "frank3_p");
    if (r) return r;
    return timed(c, NH_KCLASS_FD_CORRECT, st, [&] { return launch_fd_correct(a, st); }, "fd_correct");
}

// Stress and force from the current n and u.  after_update: the force that
// follows an FD update, whose corrector left its averaged rate in ndot (used
// for N with the n_from_rate reading).
template <typename Real>
int enqueue_force_only(nh_ctx* c, cudaStream_t st, bool after_update = false)
{
    auto a = fd_chan<Real>(c);
    a.p.n_rate = after_update && c->p.n_from_rate;
    if (c->fd_fused)
        return timed(c, NH_KCLASS_STRESS, st, [&] { return launch_fd_fused_b<Real>(a, a.n, nullptr, st); },
                     "stress_force");
    int r = NH_OK;
    if (a.P3) r = timed(c, NH_KCLASS_STRESS, st, [&] { return launch_frank3_p(a, false, st); }, "frank3_p");
    if (r) return r;
    r = timed(c, NH_KCLASS_STRESS, st, [&] { return launch_stress(a, st); }, "stress");
    if (r) return r;
    return timed(c, NH_KCLASS_FORCE, st, [&] { return launch_force(a, st); }, "force");
}

template <typename Real>
int enqueue_fd(nh_ctx* c, cudaStream_t st)
{
    auto a = fd_chan<Real>(c);
    c->bdp_step = -1;
    if (c->fd_fused) {
        // predictor + corrector: n -> nP; stress + force from nP, which is copied back into n
        int r = timed(c, NH_KCLASS_FD_PREDICT, st, [&] { return launch_fd_fused_a<Real>(a, a.n, a.nP, st); },
                      "fd_fused");
        if (r) return r;
        // after a macro LB launch of this step, the stress kernel also leaves the diagnostics' partials of
        // the updated director (with the LB launch's population, |u| and non-finite partials folded in)
        BDiag bd{};
        const bool dfold = fold_ok(c) && c->lbp_step == c->step;
        if (dfold) {
            bd.tubes = c->at<const double>(c->L.tubesd);
            bd.n_tubes = c->n_tubes;
            bd.trig = c->at<const double>(c->L.trig);
            bd.partials = c->at<double>(c->L.bpart);
            bd.lbpart = c->at<const double>(c->L.lbpart);
            bd.lbp_blocks = c->lbp_blocks;
        }
        r = timed(c, NH_KCLASS_STRESS, st,
                  [&] { return launch_fd_fused_b<Real>(a, a.nP, a.n, st, dfold ? &bd : nullptr); }, "stress_force");
        if (r) return r;
        if (dfold) {
            c->bdp_step = c->step;
            c->bdp_blocks = fd_fused_tiles(a);
            c->bdp_tubes_epoch = c->tubes_epoch;
        }
        return NH_OK;
    }
    a.p.n_rate = c->p.n_from_rate;  // the corrector keeps its averaged rate
    int r = enqueue_predict_correct_sites<Real>(c, a, st);
    if (r) return r;
    return enqueue_force_only<Real>(c, st, true);
}

template <typename Real>
int enqueue_predict_correct(nh_ctx* c, cudaStream_t st)
{
    auto a = fd_chan<Real>(c);
    if (c->fd_fused) {
        int r = timed(c, NH_KCLASS_FD_PREDICT, st, [&] { return launch_fd_fused_a<Real>(a, a.n, a.nP, st); },
                      "fd_fused");
        if (r) return r;
        return cudaMemcpyAsync(a.n, a.nP, 3 * (size_t)c->N * sizeof(Real), cudaMemcpyDeviceToDevice, st) == cudaSuccess
                   ? NH_OK
                   : fail(c, NH_ECUDA, "copy of the relaxed director");
    }
    return enqueue_predict_correct_sites<Real>(c, a, st);
}

// Relaxation with the fused kernel, alternating n -> nP -> n; an odd count
// ends with one copy back into n.
template <typename Real>
int relax_fused(nh_ctx* c, int64_t steps, cudaStream_t st)
{
    auto a = fd_chan<Real>(c);
    for (int64_t k = 0; k < steps; ++k) {
        const bool even = (k & 1) == 0;
        int r = timed(c, NH_KCLASS_FD_PREDICT, st,
                      [&] { return even ? launch_fd_fused_a<Real>(a, a.n, a.nP, st) : launch_fd_fused_a<Real>(a, a.nP, a.n, st); },
                      "fd_fused");
        if (r) return r;
    }
    if (steps & 1) NH_CUDA(c, cudaMemcpyAsync(a.n, a.nP, 3 * (size_t)c->N * sizeof(Real), cudaMemcpyDeviceToDevice, st));
    return NH_OK;
}

int enqueue_fd_any(nh_ctx* c, cudaStream_t st)
{
    return c->p.precision == NH_FP64 ? enqueue_fd<double>(c, st) : enqueue_fd<float>(c, st);
}

int enqueue_force_any(nh_ctx* c, cudaStream_t st)
{
    return c->p.precision == NH_FP64 ? enqueue_force_only<double>(c, st) : enqueue_force_only<float>(c, st);
}

// One LB step followed, when the step count reaches a multiple of dt_fd, by the FD update.
// With paper_order the FD update sits between the macroscopic fields and the
// collision of that step (Sec. II.D): a first launch writes u and rho (its
// populations are overwritten), the FD update computes the new force, and the
// step is redone from the same source buffer with the new force in the Guo
// source and u shifted by half of the old one.
int enqueue_one_step(nh_ctx* c, bool last_of_call, cudaStream_t st)
{
    const int64_t next = c->step + 1;
    const bool fd = (next % c->p.dt_fd) == 0;
    if (fd && c->p.paper_order) {
        int r = enqueue_lb(c, c->cur, true, st);
        if (r) return r;
        const size_t fbytes = 3 * (size_t)c->N * (c->p.precision == NH_FP64 ? sizeof(double) : sizeof(float));
        NH_CUDA(c, cudaMemcpyAsync(c->ws + c->L.Fprev, c->ws + c->L.F, fbytes, cudaMemcpyDeviceToDevice, st));
        r = enqueue_fd_any(c, st);
        if (r) return r;
        r = enqueue_lb(c, c->cur, false, st, true);
        if (r) return r;
        c->cur ^= 1;
        c->step = next;
        return NH_OK;
    }
    int r = enqueue_lb(c, c->cur, fd || last_of_call, st);
    if (r) return r;
    c->cur ^= 1;
    c->step = next;
    if (fd) return enqueue_fd_any(c, st);
    return NH_OK;
}

// Capture a whole dt_fd block starting from population buffer `src`.
int capture_block(nh_ctx* c, int src)
{
    const int saved_cur = c->cur;
    const int64_t saved_step = c->step;
    const int64_t saved_launches = c->launches;
    cudaStream_t cs = c->cap_stream;
    NH_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    c->cur = src;
    c->step = 0;
    int r = NH_OK;
    for (int k = 0; k < c->p.dt_fd && r == NH_OK; ++k) r = enqueue_one_step(c, false, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    const int64_t kernels = c->launches - saved_launches;
    c->cur = saved_cur;
    c->step = saved_step;
    c->launches = saved_launches;
    if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graph[src] = ex;
    c->graph_kernels[src] = kernels;
    return NH_OK;
}

int check_ready(nh_ctx* c)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (!c->bound) return fail(c, NH_ENOMEM, "no workspace bound");
    return NH_OK;
}

int set_device(nh_ctx* c)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
    if (cur != c->device) {
        e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    }
    return NH_OK;
}

template <typename Real>
int launch_store(nh_ctx* c, const void* src_dev, double* dst, int64_t count, int on_device, cudaStream_t st)
{
    if (on_device) {
        NH_CUDA(c, launch_store_vec<Real>(static_cast<const Real*>(src_dev), dst, count, st));
        c->launches += 1;
        return NH_OK;
    }
    double* stg = c->at<double>(c->L.staging);
    NH_CUDA(c, launch_store_vec<Real>(static_cast<const Real*>(src_dev), stg, count, st));
    c->launches += 1;
    NH_CUDA(c, cudaMemcpyAsync(dst, stg, count * sizeof(double), cudaMemcpyDeviceToHost, st));
    NH_CUDA(c, cudaStreamSynchronize(st));
    return NH_OK;
}

int store_field(nh_ctx* c, size_t off, double* dst, int64_t count, int on_device, cudaStream_t st)
{
    if (!dst) return NH_OK;
    const void* src = c->ws + off;
    return c->p.precision == NH_FP64 ? launch_store<double>(c, src, dst, count, on_device, st)
                                     : launch_store<float>(c, src, dst, count, on_device, st);
}

template <typename Store>
int decode_all(nh_ctx* c, double* f, int on_device, cudaStream_t st)
{
    const Store* src = c->at<const Store>(c->L.f[c->cur]);
    const float* scale = c->at<const float>(c->L.scales) + c->cur;
    double* stg = c->at<double>(c->L.staging);
    for (int i = 0; i < 19; ++i) {
        double* dst = on_device ? f + (size_t)i * c->N : stg;
        NH_CUDA(c, launch_decode_plane<Store>(src + (size_t)i * c->N, dst, c->N, scale, st));
        c->launches += 1;
        if (!on_device) {
            NH_CUDA(c, cudaMemcpyAsync(f + (size_t)i * c->N, stg, c->N * sizeof(double), cudaMemcpyDeviceToHost, st));
            NH_CUDA(c, cudaStreamSynchronize(st));
        }
    }
    return NH_OK;
}

template <typename Store>
int encode_all(nh_ctx* c, const double* f, int on_device, cudaStream_t st)
{
    Store* dst = c->at<Store>(c->L.f[c->cur]);
    const float* scale = c->at<const float>(c->L.scales) + c->cur;
    double* stg = c->at<double>(c->L.staging);
    for (int i = 0; i < 19; ++i) {
        const double* src = f + (size_t)i * c->N;
        if (!on_device) {
            NH_CUDA(c, cudaMemcpyAsync(stg, src, c->N * sizeof(double), cudaMemcpyHostToDevice, st));
            src = stg;
        }
        NH_CUDA(c, launch_encode_plane<Store>(src, dst + (size_t)i * c->N, c->N, scale, st));
        c->launches += 1;
        if (!on_device) NH_CUDA(c, cudaStreamSynchronize(st));
    }
    return NH_OK;
}

// The previous tube centroids on the device (read where the fused stress
// kernel leaves the diagnostics partials), refreshed before the next FD update
// after they changed; a pageable-memory copy, so never inside a graph capture.
int sync_tubes(nh_ctx* c, cudaStream_t st)
{
    if (!c->tubes_dirty) return NH_OK;
    NH_CUDA(c, cudaMemcpyAsync(c->ws + c->L.tubesd, c->tubes, sizeof(c->tubes), cudaMemcpyHostToDevice, st));
    c->tubes_dirty = false;
    return NH_OK;
}

int enqueue_diag(nh_ctx* c, cudaStream_t st)
{
    close_segment(c);
    DiagArgs a;
    a.f = c->ws + c->L.f[c->cur];
    a.storage = c->p.storage;
    a.shifted = c->p.shifted;
    a.n = c->ws + c->L.n;
    a.u = c->ws + c->L.u;
    a.rho = c->ws + c->L.rho;
    a.precision = c->p.precision;
    a.scale = c->at<const float>(c->L.scales) + c->cur;
    a.g = Geom{c->p.nx, c->p.ny, c->p.nz, c->p.walls_z, c->p.anchoring, c->N};
    a.K = c->p.K;
    a.q0 = c->p.q0;
    a.W0 = c->p.W0;
    a.frank3 = c->p.frank3;
    a.solid = c->has_solid ? c->at<const unsigned char>(c->L.solid) : nullptr;
    a.kd1 = c->p.frank3 ? c->p.K11 - c->p.K : 0.0;
    a.kd2 = c->p.frank3 ? c->p.K22 - c->p.K : 0.0;
    a.kd3 = c->p.frank3 ? c->p.K33 - c->p.K : 0.0;
    a.n_tubes = c->n_tubes;
    memcpy(a.tubes, c->tubes, sizeof(a.tubes));
    a.trig = c->at<const double>(c->L.trig);
    a.partials = c->at<double>(c->L.partials);
    a.result = c->at<double>(c->L.result);
    a.blocks = diag_blocks();
    if (fold_ok(c) && c->lbp_step == c->step && c->bdp_step == c->step && c->bdp_tubes_epoch == c->tubes_epoch) {
        // the fused stress kernel of this step left every partial: the final reduction alone
        NH_CUDA(c, launch_diag_final(c->at<const double>(c->L.bpart), a.result, c->bdp_blocks,
                                     diag_num_values(c->n_tubes), st));
        c->launches += 1;
        return NH_OK;
    }
    if (fold_ok(c) && c->lbp_step == c->step) {  // the last macro LB launch summed f, u and rho of this state
        a.lbpart = c->at<const double>(c->L.lbpart);
        a.lbp_blocks = c->lbp_blocks;
    }
    NH_CUDA(c, launch_diagnostics(a, st));
    c->launches += 2;
    return NH_OK;
}

}  // namespace

namespace {

// ------------------------------------------------------------ batched channels

struct BatchPlan {
    std::vector<nh_ctx*> ctxs;
    std::vector<int64_t> epochs;
    int variant = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
};

std::mutex g_batch_mu;
std::map<std::vector<nh_ctx*>, BatchPlan*> g_batch_plans;

void batch_drop_graphs(BatchPlan* b)
{
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
        b->graph_kernels[k] = 0;
    }
}

void drop_batch_plans(const nh_ctx* c)
{
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_batch_plans.begin(); it != g_batch_plans.end();) {
        if (std::find(it->first.begin(), it->first.end(), c) != it->first.end()) {
            batch_drop_graphs(it->second);
            delete it->second;
            it = g_batch_plans.erase(it);
        } else {
            ++it;
        }
    }
}

// Validate a batch and find (or build) its plan.
int batch_prepare(nh_ctx* const* ctxs, int count, int64_t n_lb_steps, BatchPlan** out)
{
    if (!ctxs || count < 1) return fail(nullptr, NH_EINVAL, "need at least one context");
    if (n_lb_steps < 0) return fail(nullptr, NH_EINVAL, "n_lb_steps must be >= 0");
    nh_ctx* c0 = ctxs[0];
    for (int k = 0; k < count; ++k) {
        nh_ctx* c = ctxs[k];
        if (!c) return fail(nullptr, NH_EINVAL, "NULL context in batch");
        if (!c->bound || !c->fields_set)
            return fail(nullptr, NH_EINVAL, "channel " + std::to_string(k) + ": workspace or fields not set");
        if (c->p.precision != c0->p.precision || c->p.storage != c0->p.storage || c->p.shifted != c0->p.shifted ||
            c->p.dt_fd != c0->p.dt_fd)
            return fail(nullptr, NH_EINVAL, "channels must share precision, storage, shifted and dt_fd");
        if (c->p.paper_order || c->p.lap_wide || c->p.n_from_rate)
            return fail(nullptr, NH_EINVAL, "channel " + std::to_string(k) +
                                                ": paper_order, lap_wide and n_from_rate are not supported in batches");
        if (c->device != c0->device) return fail(nullptr, NH_EINVAL, "channels must be on one device");
        if (c->cur != c0->cur || c->step % c0->p.dt_fd != c0->step % c0->p.dt_fd)
            return fail(nullptr, NH_EINVAL, "channels must be at the same step phase (step mod dt_fd, buffer parity)");
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c) return fail(nullptr, NH_EINVAL, "a context appears twice in the batch");
    }
    int r = set_device(c0);
    if (r) return fail(nullptr, r, c0->err);
    std::vector<nh_ctx*> key(ctxs, ctxs + count);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchPlan*& plan = g_batch_plans[key];
    std::vector<int64_t> epochs;
    for (nh_ctx* c : key) epochs.push_back(c->epoch);
    if (plan && plan->epochs != epochs) {
        batch_drop_graphs(plan);
        delete plan;
        plan = nullptr;
    }
    if (!plan) {
        plan = new (std::nothrow) BatchPlan();
        if (!plan) return fail(nullptr, NH_ENOMEM, "host allocation of the batch plan failed");
        plan->ctxs = key;
        plan->epochs = epochs;
        int v = c0->lb_variant;
        bool ok = true;
        for (nh_ctx* c : key) ok = ok && lb_variant_valid(v, c->p.nx);
        if (!ok) {  // the row-staged variant (single channels only), or a shape some channel cannot take
            v = 0;
            for (nh_ctx* c : key)
                if (!lb_variant_valid(0, c->p.nx)) v = 1;  // one site per thread fits every domain
        }
        plan->variant = v;
    }
    *out = plan;
    return NH_OK;
}

// Batch of director-only relaxations: the channels must share the precision
// and the device (their step phase is irrelevant: no LB step runs).
int batch_prepare_relax(nh_ctx* const* ctxs, int count, int64_t n_fd_steps, BatchPlan** out)
{
    if (!ctxs || count < 1) return fail(nullptr, NH_EINVAL, "need at least one context");
    if (n_fd_steps < 0) return fail(nullptr, NH_EINVAL, "n_fd_steps must be >= 0");
    nh_ctx* c0 = ctxs[0];
    for (int k = 0; k < count; ++k) {
        nh_ctx* c = ctxs[k];
        if (!c) return fail(nullptr, NH_EINVAL, "NULL context in batch");
        if (!c->bound || !c->fields_set)
            return fail(nullptr, NH_EINVAL, "channel " + std::to_string(k) + ": workspace or fields not set");
        if (c->p.precision != c0->p.precision) return fail(nullptr, NH_EINVAL, "channels must share the precision");
        if (c->p.lap_wide)
            return fail(nullptr, NH_EINVAL, "channel " + std::to_string(k) + ": lap_wide is not supported in batches");
        if (c->device != c0->device) return fail(nullptr, NH_EINVAL, "channels must be on one device");
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c) return fail(nullptr, NH_EINVAL, "a context appears twice in the batch");
    }
    int r = set_device(c0);
    if (r) return fail(nullptr, r, c0->err);
    static thread_local BatchPlan plan;
    plan.ctxs.assign(ctxs, ctxs + count);
    *out = &plan;
    return NH_OK;
}

template <typename Real, typename Store>
int batch_lb_typed(BatchPlan* b, bool write_macro, cudaStream_t st)
{
    nh_ctx* c0 = b->ctxs[0];
    const int n = (int)b->ctxs.size();
    static thread_local LBBatch<Real, Store> batch;  // large parameter block, kept off the stack
    for (int g0 = 0; g0 < n; g0 += kMaxBatch) {
        batch.count = std::min(kMaxBatch, n - g0);
        for (int k = 0; k < batch.count; ++k) batch.ch[k] = lb_chan<Real, Store>(b->ctxs[g0 + k], b->ctxs[g0 + k]->cur);
        const int grid = 8 * c0->sm_count;
        int r = timed(c0, NH_KCLASS_LB, st,
                      [&] { return launch_lb_batch(batch, c0->p.shifted != 0, write_macro, b->variant, grid, st); },
                      "lb_batch");
        if (r) return r;
    }
    return NH_OK;
}

int batch_enqueue_lb(BatchPlan* b, bool write_macro, cudaStream_t st)
{
    switch (b->ctxs[0]->p.storage) {
    case NH_STORE_F64: return batch_lb_typed<double, double>(b, write_macro, st);
    case NH_STORE_F32: return batch_lb_typed<float, float>(b, write_macro, st);
    case NH_STORE_F16S: return batch_lb_typed<float, __half>(b, write_macro, st);
    default: return batch_lb_typed<float, __nv_bfloat16>(b, write_macro, st);
    }
}

template <typename Real>
int batch_fd_typed(BatchPlan* b, cudaStream_t st, int stages = 4)
{
    nh_ctx* c0 = b->ctxs[0];
    const int n = (int)b->ctxs.size();
    static thread_local FDBatch<Real> batch;
    // the fused kernels only when every channel runs on them (not the three-constant energy, lap_wide or
    // n_from_rate, nor a channel set to the per-site kernels)
    bool fused = true, frank3 = false;
    for (nh_ctx* c : b->ctxs) {
        fused = fused && c->fd_fused;
        frank3 = frank3 || c->p.frank3;
    }
    if (fused) {
        // stages == 4: full FD update (A: n -> nP, B: nP -> F and n); stages == 2: one relaxation step (A, copy back)
        const int fstages[2] = {0, 1};
        const int classes[2] = {NH_KCLASS_FD_PREDICT, NH_KCLASS_STRESS};
        for (int k = 0; k < (stages == 4 ? 2 : 1); ++k) {
            for (int g0 = 0; g0 < n; g0 += kMaxBatch) {
                batch.count = std::min(kMaxBatch, n - g0);
                for (int j = 0; j < batch.count; ++j) batch.ch[j] = fd_chan<Real>(b->ctxs[g0 + j]);
                const int grid = 8 * c0->sm_count;
                int r = timed(c0, classes[k], st, [&] { return launch_fd_fused_batch(batch, fstages[k], grid, st); },
                              "fd_fused_batch");
                if (r) return r;
            }
        }
        if (stages != 4)
            for (nh_ctx* c : b->ctxs) {
                cudaError_t e = cudaMemcpyAsync(c->ws + c->L.n, c->ws + c->L.nP, 3 * (size_t)c->N * sizeof(Real),
                                                cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return fail(c0, NH_ECUDA, "copy of the relaxed director");
            }
        return NH_OK;
    }
    // per-site stages: predict, correct, stress, force; with the three-constant energy each of the
    // first three is preceded by the P stage of the field it differentiates (4: n, 5: n^P)
    const int classes[4] = {NH_KCLASS_FD_PREDICT, NH_KCLASS_FD_CORRECT, NH_KCLASS_STRESS, NH_KCLASS_FORCE};
    for (int stage = 0; stage < stages; ++stage) {
        const int pre = (frank3 && stage < 3) ? (stage == 1 ? 5 : 4) : -1;
        for (int pass = pre >= 0 ? 0 : 1; pass < 2; ++pass) {
            const int kernel_stage = pass == 0 ? pre : stage;
            for (int g0 = 0; g0 < n; g0 += kMaxBatch) {
                batch.count = std::min(kMaxBatch, n - g0);
                for (int k = 0; k < batch.count; ++k) batch.ch[k] = fd_chan<Real>(b->ctxs[g0 + k]);
                const int grid = 8 * c0->sm_count;
                int r = timed(c0, classes[stage], st, [&] { return launch_fd_batch(batch, kernel_stage, grid, st); },
                              "fd_batch");
                if (r) return r;
            }
        }
    }
    return NH_OK;
}

// One batched LB step (+ the batched FD update when the step count reaches a
// multiple of dt_fd) for every channel of the plan.
int batch_one_step(BatchPlan* b, bool last_of_call, cudaStream_t st)
{
    nh_ctx* c0 = b->ctxs[0];
    const int64_t next = c0->step + 1;
    const bool fd = (next % c0->p.dt_fd) == 0;
    int r = batch_enqueue_lb(b, fd || last_of_call, st);
    if (r) return r;
    for (nh_ctx* c : b->ctxs) {
        c->cur ^= 1;
        c->step += 1;
    }
    if (fd) return c0->p.precision == NH_FP64 ? batch_fd_typed<double>(b, st) : batch_fd_typed<float>(b, st);
    return NH_OK;
}

int batch_capture(BatchPlan* b, int parity)
{
    nh_ctx* c0 = b->ctxs[0];
    std::vector<int> cur;
    std::vector<int64_t> step;
    for (nh_ctx* c : b->ctxs) {
        cur.push_back(c->cur);
        step.push_back(c->step);
        c->cur = parity;
        c->step = 0;
    }
    const int64_t saved_launches = c0->launches;
    cudaStream_t cs = c0->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int r = e == cudaSuccess ? NH_OK : cuda_fail(c0, e, "cudaStreamBeginCapture");
    if (r == NH_OK) {
        for (int k = 0; k < c0->p.dt_fd && r == NH_OK; ++k) r = batch_one_step(b, false, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (r == NH_OK && e != cudaSuccess) r = cuda_fail(c0, e, "cudaStreamEndCapture");
        if (r == NH_OK) {
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            if (e != cudaSuccess)
                r = cuda_fail(c0, e, "cudaGraphInstantiate");
            else {
                b->graph[parity] = ex;
                b->graph_kernels[parity] = c0->launches - saved_launches;
            }
        }
        if (g) cudaGraphDestroy(g);
    }
    c0->launches = saved_launches;
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
        b->ctxs[k]->cur = cur[k];
        b->ctxs[k]->step = step[k];
    }
    return r;
}

// ------------------------------------------------------------ slabs along y

// Halo plan of `count` slabs stacked along y (slab k below slab k + 1, the
// last below the first: periodic).  Slab k has interior rows 1 .. ny[k] and
// ghost rows 0 and ny[k] + 1.  Its lower ghost row is the last interior row of
// the slab below, its upper ghost row the first interior row of the slab
// above.  Populations: only the planes the interior pulls across each face,
// e_y = +1 (3, 7, 10, 15, 17) from below and e_y = -1 (4, 8, 9, 16, 18) from
// above; fields: every component.
int slab_plan(int count, const int32_t* ny, int kind, std::vector<nh_row_copy>& out)
{
    if (count < 1 || count > kMaxSlabs || !ny) return NH_EINVAL;
    if (kind != NH_HALO_POPULATIONS && kind != NH_HALO_VECTOR && kind != NH_HALO_STRESS) return NH_EINVAL;
    for (int k = 0; k < count; ++k)
        if (ny[k] < 1) return NH_EINVAL;
    const uint32_t up = (1u << 3) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 17);
    const uint32_t down = (1u << 4) | (1u << 8) | (1u << 9) | (1u << 16) | (1u << 18);
    const uint32_t all = kind == NH_HALO_VECTOR ? 0x7u : 0x1FFu;
    out.clear();
    for (int k = 0; k < count; ++k) {
        const int below = (k + count - 1) % count, above = (k + 1) % count;
        out.push_back(nh_row_copy{below, ny[below], k, 0, kind == NH_HALO_POPULATIONS ? up : all});
        out.push_back(nh_row_copy{above, 1, k, ny[k] + 1, kind == NH_HALO_POPULATIONS ? down : all});
    }
    return NH_OK;
}

// Enqueue the row copies of a plan on one workspace region of every slab
// (the field `field` of each slab's own layout, or with populations the
// buffer each slab wrote last; elements of elem bytes, component c of slab k
// at c * N_k).
int slab_copy(nh_ctx* const* slabs, int count, int kind, size_t Layout::*field, bool populations, int elem,
              cudaStream_t st)
{
    std::vector<int32_t> ny(count);
    for (int k = 0; k < count; ++k) ny[k] = slabs[k]->p.ny - 2;
    std::vector<nh_row_copy> plan;
    int r = slab_plan(count, ny.data(), kind, plan);
    if (r) return fail(nullptr, r, "slab plan");
    static thread_local RowCopyList list;
    list.count = 0;
    auto flush = [&]() -> int {
        cudaError_t e = launch_row_copies(list, elem, st);
        slabs[0]->launches += list.count > 0 ? 1 : 0;
        list.count = 0;
        return e == cudaSuccess ? NH_OK : fail(nullptr, NH_ECUDA, std::string("row copies: ") + cudaGetErrorString(e));
    };
    for (const nh_row_copy& c : plan) {
        nh_ctx* a = slabs[c.src_slab];
        nh_ctx* b = slabs[c.dst_slab];
        const size_t oa = populations ? a->L.f[a->cur] : a->L.*field;
        const size_t ob = populations ? b->L.f[b->cur] : b->L.*field;
        const int nx = a->p.nx, nz = a->p.nz;
        for (int comp = 0; comp < 19; ++comp) {
            if (!(c.comp_mask >> comp & 1u)) continue;
            RowCopyItem it;
            const int first = populations ? comp : 0;  // populations: one plane per item; fields: all components
            it.src = a->ws + oa + ((size_t)first * a->N + (size_t)nx * c.src_row) * elem;
            it.dst = b->ws + ob + ((size_t)first * b->N + (size_t)nx * c.dst_row) * elem;
            it.nx = nx;
            it.nz = nz;
            it.comps = populations ? 1 : (kind == NH_HALO_VECTOR ? 3 : 9);
            it.src_zstride = nx * a->p.ny;
            it.dst_zstride = nx * b->p.ny;
            it.src_cstride = a->N;
            it.dst_cstride = b->N;
            list.item[list.count++] = it;
            if (list.count == kMaxRowCopies && (r = flush())) return r;
            if (!populations) break;
        }
    }
    return flush();
}

int slab_validate(nh_ctx* const* slabs, int count)
{
    if (!slabs || count < 1 || count > kMaxSlabs) return fail(nullptr, NH_EINVAL, "need 1 to 64 slabs");
    nh_ctx* c0 = slabs[0];
    for (int k = 0; k < count; ++k) {
        nh_ctx* c = slabs[k];
        if (!c) return fail(nullptr, NH_EINVAL, "NULL slab");
        if (!c->bound || !c->fields_set)
            return fail(nullptr, NH_EINVAL, "slab " + std::to_string(k) + ": workspace or fields not set");
        if (c->p.ny < 3) return fail(nullptr, NH_EINVAL, "a slab needs ny >= 3 (two ghost rows and an interior row)");
        nh_params a = c->p, b = c0->p;
        a.ny = b.ny = 0;
        if (memcmp(&a, &b, sizeof(a)) != 0)
            return fail(nullptr, NH_EINVAL, "slabs must share every parameter but ny");
        if (c->p.paper_order || c->p.frank3 || c->p.lap_wide || c->has_solid)
            return fail(nullptr, NH_EINVAL, "paper_order, frank3, lap_wide and obstacles are not supported in slabs");
        if (c->p.storage != NH_STORE_F64 && c->p.storage != NH_STORE_F32)
            return fail(nullptr, NH_EINVAL, "slabs exchange raw populations: F64 or F32 stores only");
        if (c->device != c0->device) return fail(nullptr, NH_EINVAL, "slabs must be on one device");
        if (c->cur != c0->cur || c->step != c0->step)
            return fail(nullptr, NH_EINVAL, "slabs must be at the same step and buffer parity");
        for (int j = 0; j < k; ++j)
            if (slabs[j] == c) return fail(nullptr, NH_EINVAL, "a context appears twice among the slabs");
    }
    return set_device(c0);
}

// Stress of every slab, sigma halo, force of every slab (per-site kernels).
template <typename Real>
int slab_force(nh_ctx* const* slabs, int count, bool after_update, cudaStream_t st)
{
    for (int k = 0; k < count; ++k) {
        auto a = fd_chan<Real>(slabs[k]);
        a.p.n_rate = after_update && slabs[k]->p.n_from_rate;
        NH_CUDA(slabs[0], launch_stress(a, st));
        slabs[k]->launches += 1;
    }
    int r = slab_copy(slabs, count, NH_HALO_STRESS, &Layout::sigma, false, sizeof(Real), st);
    if (r) return r;
    for (int k = 0; k < count; ++k) {
        NH_CUDA(slabs[0], launch_force(fd_chan<Real>(slabs[k]), st));
        slabs[k]->launches += 1;
    }
    return NH_OK;
}

// One FD update of every slab with the halo exchanges between the stages.
template <typename Real>
int slab_fd(nh_ctx* const* slabs, int count, cudaStream_t st)
{
    const int E = sizeof(Real);
    int r = slab_copy(slabs, count, NH_HALO_VECTOR, &Layout::u, false, E, st);
    for (int k = 0; k < count && !r; ++k) {
        NH_CUDA(slabs[0], launch_fd_predict(fd_chan<Real>(slabs[k]), st));
        slabs[k]->launches += 1;
    }
    if (!r) r = slab_copy(slabs, count, NH_HALO_VECTOR, &Layout::nP, false, E, st);
    for (int k = 0; k < count && !r; ++k) {
        auto a = fd_chan<Real>(slabs[k]);
        a.p.n_rate = slabs[k]->p.n_from_rate;
        NH_CUDA(slabs[0], launch_fd_correct(a, st));
        slabs[k]->launches += 1;
    }
    if (!r) r = slab_copy(slabs, count, NH_HALO_VECTOR, &Layout::n, false, E, st);
    if (!r) r = slab_force<Real>(slabs, count, true, st);
    return r;
}

}  // namespace

extern "C" {

int nh_slab_plan(int count, const int32_t* ny_local, int kind, nh_row_copy* out, int capacity, int* n_out)
{
    std::vector<nh_row_copy> plan;
    int r = slab_plan(count, ny_local, kind, plan);
    if (r) return fail(nullptr, r, "nh_slab_plan: need 1 to 64 slabs with ny_local >= 1 and a known kind");
    if (n_out) *n_out = (int)plan.size();
    if (out) {
        if (capacity < (int)plan.size()) return fail(nullptr, NH_EINVAL, "nh_slab_plan: capacity too small");
        std::copy(plan.begin(), plan.end(), out);
    }
    return NH_OK;
}

int nh_slab_init(nh_ctx* const* slabs, int count, void* stream)
{
    NvtxRange range_("nh_slab_init");
    int r = slab_validate(slabs, count);
    if (r) return r;
    nh_ctx* c0 = slabs[0];
    cudaStream_t st = pick(c0, stream);
    const int E = (int)real_size(c0->p);
    const int S = (int)store_size(c0->p);
    if ((r = slab_copy(slabs, count, NH_HALO_POPULATIONS, nullptr, true, S, st))) return r;
    if ((r = slab_copy(slabs, count, NH_HALO_VECTOR, &Layout::n, false, E, st))) return r;
    if ((r = slab_copy(slabs, count, NH_HALO_VECTOR, &Layout::u, false, E, st))) return r;
    r = c0->p.precision == NH_FP64 ? slab_force<double>(slabs, count, false, st) : slab_force<float>(slabs, count, false, st);
    if (r) return fail(nullptr, r, "nh_slab_init: " + std::string(nh_last_error(nullptr)));
    return NH_OK;
}

int nh_slab_step(nh_ctx* const* slabs, int count, int64_t n_lb_steps, void* stream)
{
    NvtxRange range_("nh_slab_step");
    int r = slab_validate(slabs, count);
    if (r) return r;
    if (n_lb_steps < 0) return fail(nullptr, NH_EINVAL, "n_lb_steps must be >= 0");
    nh_ctx* c0 = slabs[0];
    cudaStream_t st = pick(c0, stream);
    const int E = (int)real_size(c0->p);
    const int S = (int)store_size(c0->p);
    for (int64_t s = 0; s < n_lb_steps; ++s) {
        const int64_t next = c0->step + 1;
        const bool fd = (next % c0->p.dt_fd) == 0;
        const bool last = s + 1 == n_lb_steps;
        for (int k = 0; k < count; ++k) {
            if ((r = enqueue_lb(slabs[k], slabs[k]->cur, fd || last, st))) return fail(nullptr, r, slabs[k]->err);
            slabs[k]->cur ^= 1;
            slabs[k]->step = next;
        }
        if ((r = slab_copy(slabs, count, NH_HALO_POPULATIONS, nullptr, true, S, st))) return r;
        if (fd) {
            r = c0->p.precision == NH_FP64 ? slab_fd<double>(slabs, count, st) : slab_fd<float>(slabs, count, st);
            if (r) return fail(nullptr, r, "nh_slab_step: " + std::string(nh_last_error(nullptr)) + c0->err);
        } else if (last) {
            if ((r = slab_copy(slabs, count, NH_HALO_VECTOR, &Layout::u, false, E, st))) return r;
        }
    }
    for (int k = 0; k < count; ++k) close_segment(slabs[k]);
    return NH_OK;
}

const char* nh_error_string(int code)
{
    switch (code) {
    case NH_OK: return "ok";
    case NH_EINVAL: return "invalid argument";
    case NH_ECUDA: return "CUDA error";
    case NH_ENOMEM: return "workspace missing or too small";
    case NH_EUNSTABLE: return "non-finite values in the fields";
    case NH_ETIMEOUT: return "bounded wait expired";
    default: return "unknown error";
    }
}

const char* nh_last_error(const nh_ctx* ctx) { return ctx ? ctx->err.c_str() : g_global_err.c_str(); }

int nh_workspace_bytes(const nh_params* p, size_t* bytes)
{
    std::string err;
    int r = validate(p, err);
    if (r) return fail(nullptr, r, err);
    if (!bytes) return fail(nullptr, NH_EINVAL, "bytes is NULL");
    *bytes = make_layout(*p).total;
    return NH_OK;
}

int nh_create(const nh_params* p, void* cuda_stream, nh_ctx** out)
{
    if (!out) return fail(nullptr, NH_EINVAL, "out is NULL");
    *out = nullptr;
    std::string err;
    int r = validate(p, err);
    if (r) return fail(nullptr, r, err);
    nh_ctx* c = new (std::nothrow) nh_ctx();
    if (!c) return fail(nullptr, NH_ENOMEM, "host allocation of the context failed");
    c->p = *p;
    c->N = p->nx * p->ny * p->nz;
    c->lb_variant = lb_variant_valid(0, p->nx) ? 0 : 1;
    // the three-constant correction, the wide Laplacian and N from the rate run on the per-site FD kernels
    if (p->frank3 || p->lap_wide || p->n_from_rate) c->fd_fused = 0;
    c->L = make_layout(*p);
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        fail(nullptr, NH_ECUDA, std::string("nh_create: ") + cudaGetErrorString(e));
        delete c;
        return NH_ECUDA;
    }
    *out = c;
    return NH_OK;
}

int nh_bind_workspace(nh_ctx* c, void* dev_ptr, size_t bytes)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (!dev_ptr) return fail(c, NH_EINVAL, "workspace pointer is NULL");
    if (reinterpret_cast<uintptr_t>(dev_ptr) % kAlign) return fail(c, NH_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < c->L.total)
        return fail(c, NH_ENOMEM, "workspace too small: need " + std::to_string(c->L.total) + " bytes");
    drop_graphs(c);
    c->ws = static_cast<char*>(dev_ptr);
    c->ws_bytes = bytes;
    {
        int r = set_device(c);
        if (r) return r;
        NH_CUDA(c, launch_trig_table(c->at<double>(c->L.trig), c->p.nx, c->p.ny, c->stream));
        c->launches += 1;
        NH_CUDA(c, lb_rows_prepare(c->p.nx, c->p.storage));  // the row-staged LB kernel of 16-bit stores
    }
    c->bound = true;
    c->lbp_step = -1;
    c->bdp_step = -1;
    c->fields_set = false;
    c->cur = 0;
    c->step = 0;
    return NH_OK;
}

int nh_set_fields(nh_ctx* c, const double* n, const double* u, const double* rho, int on_device)
{
    NvtxRange range_("nh_set_fields");
    int r = check_ready(c);
    if (r) return r;
    if (!n) return fail(c, NH_EINVAL, "director n is required");
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->stream;
    const size_t N = c->N;
    const double *dn = n, *du = u, *drho = rho;
    if (!on_device) {
        double* stg = c->at<double>(c->L.staging);
        NH_CUDA(c, cudaMemcpyAsync(stg, n, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st));
        dn = stg;
        if (u) {
            NH_CUDA(c, cudaMemcpyAsync(stg + 3 * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st));
            du = stg + 3 * N;
        }
        if (rho) {
            NH_CUDA(c, cudaMemcpyAsync(stg + 6 * N, rho, N * sizeof(double), cudaMemcpyHostToDevice, st));
            drho = stg + 6 * N;
        }
    }
    // 16-bit stores: scales start at 1 until the probe below sets them
    const float ones[4] = {1.f, 1.f, 1.f, 1.f};
    NH_CUDA(c, cudaMemcpyAsync(c->ws + c->L.scales, ones, sizeof(ones), cudaMemcpyHostToDevice, st));
    NH_CUDA(c, cudaMemsetAsync(c->ws + c->L.absmax, 0, 4 * sizeof(float), st));
    c->cur = 0;
    c->step = 0;
    if (c->p.precision == NH_FP64) {
        NH_CUDA(c, launch_load_fields<double>(dn, du, drho, c->at<double>(c->L.n), c->at<double>(c->L.u),
                                              c->at<double>(c->L.rho), c->N, st));
    } else {
        NH_CUDA(c, launch_load_fields<float>(dn, du, drho, c->at<float>(c->L.n), c->at<float>(c->L.u),
                                             c->at<float>(c->L.rho), c->N, st));
    }
    c->launches += 1;
    // LC force of the initial fields (Eq. force-lc-eq)
    r = enqueue_force_any(c, st);
    if (r) return r;
    // equilibrium populations
    if (c->p.precision == NH_FP64) {
        NH_CUDA(c, launch_init_populations<double, double>(c->at<double>(c->L.rho), c->at<double>(c->L.u),
                                                           c->at<double>(c->L.f[0]), c->at<float>(c->L.scales),
                                                           c->N, c->p.shifted != 0, st));
    } else {
        float* sc = c->at<float>(c->L.scales);
        if (c->p.storage != NH_STORE_F32) {
            NH_CUDA(c, launch_scale_init(c->at<float>(c->L.rho), c->at<float>(c->L.u), c->at<float>(c->L.F), c->p.g,
                                         c->N, sc, c->at<unsigned>(c->L.absmax), st));
            c->launches += 2;
        }
        switch (c->p.storage) {
        case NH_STORE_F32:
            NH_CUDA(c, launch_init_populations<float, float>(c->at<float>(c->L.rho), c->at<float>(c->L.u),
                                                             c->at<float>(c->L.f[0]), sc, c->N, c->p.shifted != 0,
                                                             st));
            break;
        case NH_STORE_F16S:
            NH_CUDA(c, launch_init_populations<float, __half>(c->at<float>(c->L.rho), c->at<float>(c->L.u),
                                                              c->at<__half>(c->L.f[0]), sc, c->N, true, st));
            break;
        default:
            NH_CUDA(c, launch_init_populations<float, __nv_bfloat16>(c->at<float>(c->L.rho), c->at<float>(c->L.u),
                                                                     c->at<__nv_bfloat16>(c->L.f[0]), sc, c->N,
                                                                     true, st));
            break;
        }
    }
    c->launches += 1;
    if (!on_device) NH_CUDA(c, cudaStreamSynchronize(st));
    c->fields_set = true;
    c->snap_valid = false;
    c->lbp_step = -1;
    c->bdp_step = -1;
    return NH_OK;
}

int nh_get_fields(nh_ctx* c, double* n, double* u, double* rho, int on_device)
{
    int r = check_ready(c);
    if (r) return r;
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->stream;
    if ((r = bounded_wait(c, st))) return r;
    if ((r = store_field(c, c->L.n, n, 3 * (int64_t)c->N, on_device, st))) return r;
    if ((r = store_field(c, c->L.u, u, 3 * (int64_t)c->N, on_device, st))) return r;
    if ((r = store_field(c, c->L.rho, rho, (int64_t)c->N, on_device, st))) return r;
    NH_CUDA(c, cudaStreamSynchronize(st));
    return NH_OK;
}

int nh_get_force(nh_ctx* c, double* F, int on_device)
{
    int r = check_ready(c);
    if (r) return r;
    if ((r = set_device(c))) return r;
    if ((r = bounded_wait(c, c->stream))) return r;
    if ((r = store_field(c, c->L.F, F, 3 * (int64_t)c->N, on_device, c->stream))) return r;
    NH_CUDA(c, cudaStreamSynchronize(c->stream));
    return NH_OK;
}

int nh_get_populations(nh_ctx* c, double* f, int on_device)
{
    int r = check_ready(c);
    if (r) return r;
    if (!f) return fail(c, NH_EINVAL, "f is NULL");
    if ((r = set_device(c))) return r;
    if ((r = bounded_wait(c, c->stream))) return r;
    switch (c->p.storage) {
    case NH_STORE_F64: r = decode_all<double>(c, f, on_device, c->stream); break;
    case NH_STORE_F32: r = decode_all<float>(c, f, on_device, c->stream); break;
    case NH_STORE_F16S: r = decode_all<__half>(c, f, on_device, c->stream); break;
    default: r = decode_all<__nv_bfloat16>(c, f, on_device, c->stream); break;
    }
    if (r) return r;
    NH_CUDA(c, cudaStreamSynchronize(c->stream));
    return NH_OK;
}

int nh_set_populations(nh_ctx* c, const double* f, int on_device)
{
    int r = check_ready(c);
    if (r) return r;
    if (!f) return fail(c, NH_EINVAL, "f is NULL");
    if ((r = set_device(c))) return r;
    switch (c->p.storage) {
    case NH_STORE_F64: r = encode_all<double>(c, f, on_device, c->stream); break;
    case NH_STORE_F32: r = encode_all<float>(c, f, on_device, c->stream); break;
    case NH_STORE_F16S: r = encode_all<__half>(c, f, on_device, c->stream); break;
    default: r = encode_all<__nv_bfloat16>(c, f, on_device, c->stream); break;
    }
    if (r) return r;
    c->lbp_step = -1;
    c->bdp_step = -1;
    NH_CUDA(c, cudaStreamSynchronize(c->stream));
    return NH_OK;
}

int nh_restore(nh_ctx* c, const double* n, const double* F, const double* u, const double* rho, int64_t step,
               int on_device)
{
    int r = check_ready(c);
    if (r) return r;
    if (!n) return fail(c, NH_EINVAL, "director n is required");
    if (step < 0) return fail(c, NH_EINVAL, "step must be >= 0");
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->stream;
    const size_t N = c->N;
    const size_t R = real_size(c->p);
    double* stg = c->at<double>(c->L.staging);
    // load n (exact, no renormalisation), u, rho and F by staging through FP64
    struct Item {
        const double* src;
        size_t off;
        size_t count;
    } items[4] = {{n, c->L.n, 3 * N}, {u, c->L.u, 3 * N}, {rho, c->L.rho, N}, {F, c->L.F, 3 * N}};
    for (auto& it : items) {
        if (!it.src) continue;
        const double* src = it.src;
        if (!on_device) {
            NH_CUDA(c, cudaMemcpyAsync(stg, src, it.count * sizeof(double), cudaMemcpyHostToDevice, st));
            src = stg;
        }
        if (R == 8) {
            NH_CUDA(c, cudaMemcpyAsync(c->ws + it.off, src, it.count * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            // narrow to float with the encode kernel of the F32 store (plain conversion, scale unused)
            for (size_t k = 0; k < it.count; k += N)
                NH_CUDA(c, launch_encode_plane<float>(src + k, c->at<float>(it.off) + k, c->N,
                                                      c->at<const float>(c->L.scales), st));
        }
        if (!on_device) NH_CUDA(c, cudaStreamSynchronize(st));
    }
    if (!F) {
        r = enqueue_force_any(c, st);
        if (r) return r;
    }
    c->step = step;
    c->fields_set = true;
    c->snap_valid = false;
    c->lbp_step = -1;
    c->bdp_step = -1;
    NH_CUDA(c, cudaStreamSynchronize(st));
    return NH_OK;
}

int nh_step(nh_ctx* c, int64_t n_lb_steps, void* stream)
{
    NvtxRange range_("nh_step");
    int r = check_ready(c);
    if (r) return r;
    if (!c->fields_set) return fail(c, NH_EINVAL, "nh_set_fields must be called before nh_step");
    if (n_lb_steps < 0) return fail(c, NH_EINVAL, "n_lb_steps must be >= 0");
    if ((r = set_device(c))) return r;
    cudaStream_t st = pick(c, stream);
    if ((r = sync_tubes(c, st))) return r;
    const int dt = c->p.dt_fd;
    int64_t left = n_lb_steps;
    while (left > 0) {
        if (c->use_graphs && !c->timing && c->step % dt == 0 && left >= dt) {
            if (!c->graph[c->cur]) {
                r = capture_block(c, c->cur);
                if (r) return r;
            }
            NH_CUDA(c, cudaGraphLaunch(c->graph[c->cur], st));
            c->launches += c->graph_kernels[c->cur];
            if (dt & 1) c->cur ^= 1;
            c->step += dt;
            left -= dt;
            if (fold_ok(c)) {  // the block ends with a macro LB launch (an FD step)
                c->lbp_step = c->step;
                c->lbp_blocks = lb_blocks(c->lb_variant, c->N);
                c->bdp_step = -1;
                if (c->fd_fused) {  // ... and its fused stress kernel left the director's partials
                    c->bdp_step = c->step;
                    c->bdp_blocks = c->p.precision == NH_FP64 ? fd_fused_tiles(fd_chan<double>(c))
                                                             : fd_fused_tiles(fd_chan<float>(c));
                    c->bdp_tubes_epoch = c->tubes_epoch;
                }
            } else {
                c->bdp_step = -1;
            }
        } else {
            r = enqueue_one_step(c, left == 1, st);
            if (r) return r;
            left -= 1;
        }
    }
    close_segment(c);
    return NH_OK;
}

int nh_fd_update(nh_ctx* c, void* stream)
{
    NvtxRange range_("nh_fd_update");
    int r = check_ready(c);
    if (r) return r;
    if (!c->fields_set) return fail(c, NH_EINVAL, "nh_set_fields must be called before nh_fd_update");
    if ((r = set_device(c))) return r;
    if ((r = sync_tubes(c, pick(c, stream)))) return r;
    r = enqueue_fd_any(c, pick(c, stream));
    close_segment(c);
    return r;
}

int nh_batch_step(nh_ctx* const* ctxs, int count, int64_t n_lb_steps, void* stream)
{
    NvtxRange range_("nh_batch_step");
    BatchPlan* plan = nullptr;
    int r = batch_prepare(ctxs, count, n_lb_steps, &plan);
    if (r) return r;
    nh_ctx* c0 = ctxs[0];
    cudaStream_t st = pick(c0, stream);
    const int dt = c0->p.dt_fd;
    int64_t left = n_lb_steps;
    while (left > 0) {
        if (c0->use_graphs && !c0->timing && c0->step % dt == 0 && left >= dt) {
            const int parity = c0->cur;
            if (!plan->graph[parity]) {
                r = batch_capture(plan, parity);
                if (r) return fail(nullptr, r, "batch graph capture: " + c0->err);
            }
            cudaError_t e = cudaGraphLaunch(plan->graph[parity], st);
            if (e != cudaSuccess) return fail(nullptr, NH_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
            c0->launches += plan->graph_kernels[parity];
            for (nh_ctx* c : plan->ctxs) {
                if (dt & 1) c->cur ^= 1;
                c->step += dt;
            }
            left -= dt;
        } else {
            r = batch_one_step(plan, left == 1, st);
            if (r) return fail(nullptr, r, "batch step: " + c0->err);
            left -= 1;
        }
    }
    close_segment(c0);
    return NH_OK;
}

int nh_batch_autotune(nh_ctx* const* ctxs, int count, void* stream, int* chosen)
{
    BatchPlan* plan = nullptr;
    int r = batch_prepare(ctxs, count, 1, &plan);
    if (r) return r;
    nh_ctx* c0 = ctxs[0];
    cudaStream_t st = pick(c0, stream);
    close_segment(c0);
    const int saved_timing = c0->timing;
    c0->timing = 0;
    cudaEvent_t e0 = get_event(c0), e1 = get_event(c0);
    float best_ms = 1e30f;
    int best = plan->variant;
    const int saved = plan->variant;
    for (int v = 0; v < kLBVariantCount && r == NH_OK; ++v) {
        bool ok = true;
        for (nh_ctx* c : plan->ctxs) ok = ok && lb_variant_valid(v, c->p.nx);
        if (!ok) continue;
        plan->variant = v;
        r = batch_enqueue_lb(plan, false, st);  // streams the current buffers into the others, no swap
        if (r) break;
        cudaEventRecord(e0, st);
        for (int k = 0; k < 5 && r == NH_OK; ++k) r = batch_enqueue_lb(plan, false, st);
        cudaEventRecord(e1, st);
        if (r) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            r = fail(nullptr, NH_ECUDA, "cudaEventSynchronize");
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    c0->free_events.push_back(e0);
    c0->free_events.push_back(e1);
    c0->timing = saved_timing;
    plan->variant = best;
    if (best != saved) batch_drop_graphs(plan);
    if (chosen) *chosen = best;
    return r;
}

int nh_relax(nh_ctx* c, int64_t n_fd_steps, void* stream)
{
    NvtxRange range_("nh_relax");
    int r = check_ready(c);
    if (r) return r;
    if (!c->fields_set) return fail(c, NH_EINVAL, "nh_set_fields must be called before nh_relax");
    if (n_fd_steps < 0) return fail(c, NH_EINVAL, "n_fd_steps must be >= 0");
    if ((r = set_device(c))) return r;
    cudaStream_t st = pick(c, stream);
    c->lbp_step = -1;  // u is cleared
    c->bdp_step = -1;
    NH_CUDA(c, cudaMemsetAsync(c->ws + c->L.u, 0, 3 * (size_t)c->N * real_size(c->p), st));
    if (c->fd_fused) {
        r = c->p.precision == NH_FP64 ? relax_fused<double>(c, n_fd_steps, st) : relax_fused<float>(c, n_fd_steps, st);
    } else {
        for (int64_t k = 0; k < n_fd_steps && r == NH_OK; ++k)
            r = c->p.precision == NH_FP64 ? enqueue_predict_correct<double>(c, st)
                                          : enqueue_predict_correct<float>(c, st);
    }
    close_segment(c);
    return r;
}

int nh_batch_relax(nh_ctx* const* ctxs, int count, int64_t n_fd_steps, void* stream)
{
    NvtxRange range_("nh_batch_relax");
    BatchPlan* plan = nullptr;
    int r = batch_prepare_relax(ctxs, count, n_fd_steps, &plan);
    if (r) return r;
    nh_ctx* c0 = ctxs[0];
    cudaStream_t st = pick(c0, stream);
    for (nh_ctx* c : plan->ctxs) {
        c->lbp_step = -1;  // u is cleared
        c->bdp_step = -1;
        cudaError_t e = cudaMemsetAsync(c->ws + c->L.u, 0, 3 * (size_t)c->N * real_size(c->p), st);
        if (e != cudaSuccess) return fail(nullptr, NH_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    }
    for (int64_t k = 0; k < n_fd_steps && r == NH_OK; ++k)
        r = c0->p.precision == NH_FP64 ? batch_fd_typed<double>(plan, st, 2) : batch_fd_typed<float>(plan, st, 2);
    close_segment(c0);
    if (r) return fail(nullptr, r, "batch relax: " + c0->err);
    return NH_OK;
}

int nh_director_change(nh_ctx* c, double* max_change)
{
    int r = check_ready(c);
    if (r) return r;
    if (!max_change) return fail(c, NH_EINVAL, "max_change is NULL");
    if (!c->fields_set) return fail(c, NH_EINVAL, "nh_set_fields must be called before nh_director_change");
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->stream;
    if ((r = bounded_wait(c, st))) return r;
    double* out = c->at<double>(c->L.result);
    double* partial = c->at<double>(c->L.partials);
    if (c->p.precision == NH_FP64)
        NH_CUDA(c, launch_director_change<double>(c->at<double>(c->L.n), c->at<double>(c->L.snap), partial, out, c->N, st));
    else
        NH_CUDA(c, launch_director_change<float>(c->at<float>(c->L.n), c->at<float>(c->L.snap), partial, out, c->N, st));
    c->launches += 2;
    double v = 0.0;
    NH_CUDA(c, cudaMemcpyAsync(&v, out, sizeof(double), cudaMemcpyDeviceToHost, st));
    NH_CUDA(c, cudaStreamSynchronize(st));
    *max_change = c->snap_valid ? v : INFINITY;
    c->snap_valid = true;
    return NH_OK;
}

int nh_symmetrize_c4(nh_ctx* c)
{
    int r = check_ready(c);
    if (r) return r;
    if (!c->fields_set) return fail(c, NH_EINVAL, "nh_set_fields must be called before nh_symmetrize_c4");
    if (c->p.nx != c->p.ny) return fail(c, NH_EINVAL, "C4 symmetrisation needs nx == ny");
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->stream;
    const size_t bytes = 3 * (size_t)c->N * real_size(c->p);
    if (c->p.precision == NH_FP64)
        NH_CUDA(c, launch_symmetrize_c4<double>(c->at<double>(c->L.n), c->at<double>(c->L.nP), c->p.nx, c->p.nz, st));
    else
        NH_CUDA(c, launch_symmetrize_c4<float>(c->at<float>(c->L.n), c->at<float>(c->L.nP), c->p.nx, c->p.nz, st));
    c->launches += 1;
    NH_CUDA(c, cudaMemcpyAsync(c->ws + c->L.n, c->ws + c->L.nP, bytes, cudaMemcpyDeviceToDevice, st));
    c->bdp_step = -1;  // the director changed
    return NH_OK;
}

int nh_set_solid(nh_ctx* c, const uint8_t* mask, int on_device)
{
    int r = check_ready(c);
    if (r) return r;
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->stream;
    drop_graphs(c);
    c->lbp_step = -1;
    c->bdp_step = -1;
    if (!mask) {
        c->has_solid = false;
    } else {
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        NH_CUDA(c, cudaMemcpyAsync(c->ws + c->L.solid, mask, (size_t)c->N, kind, st));
        // fluid-site count (the shifted store's rho0 = 1 per fluid site in the mass)
        std::vector<uint8_t> host((size_t)c->N);
        NH_CUDA(c, cudaMemcpyAsync(host.data(), c->ws + c->L.solid, (size_t)c->N, cudaMemcpyDeviceToHost, st));
        NH_CUDA(c, cudaStreamSynchronize(st));
        int64_t fluid = 0;
        for (uint8_t b : host) fluid += b == 0;
        c->n_fluid = fluid;
        c->has_solid = true;
    }
    if (c->fields_set) {  // the stress, and so the force, depend on the obstacles
        r = enqueue_force_any(c, st);
        if (r) return r;
        close_segment(c);
    }
    return NH_OK;
}

int nh_set_tubes(nh_ctx* c, const double* centres, int count)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (count < 0 || count > NH_MAX_TUBES) return fail(c, NH_EINVAL, "tube count out of range");
    if (count > 0 && !centres) return fail(c, NH_EINVAL, "centres is NULL");
    if (count != c->n_tubes) drop_graphs(c);  // a captured stress kernel carries the tube count
    c->n_tubes = count;
    for (int k = 0; k < count; ++k) {
        c->tubes[k][0] = centres[2 * k];
        c->tubes[k][1] = centres[2 * k + 1];
    }
    c->tubes_dirty = true;
    c->tubes_epoch += 1;
    return NH_OK;
}

int nh_diagnostics_enqueue(nh_ctx* c, void* stream)
{
    NvtxRange range_("nh_diagnostics_enqueue");
    int r = check_ready(c);
    if (r) return r;
    if ((r = set_device(c))) return r;
    cudaStream_t st = pick(c, stream);
    if ((r = enqueue_diag(c, st))) return r;
    c->diag_stream = st;
    c->diag_tubes = c->n_tubes;
    c->diag_pending = true;
    return NH_OK;
}

int nh_diagnostics_read(nh_ctx* c, nh_diag* out)
{
    int r = check_ready(c);
    if (r) return r;
    if (!out) return fail(c, NH_EINVAL, "out is NULL");
    if (!c->diag_pending) return fail(c, NH_EINVAL, "no diagnostics enqueued");
    if ((r = set_device(c))) return r;
    cudaStream_t st = c->diag_stream;
    if ((r = bounded_wait(c, st))) return r;  // the result stays pending: a later call reads it
    const int V = diag_num_values(c->diag_tubes);
    NH_CUDA(c, cudaMemcpyAsync(c->host_result, c->ws + c->L.result, V * sizeof(double), cudaMemcpyDeviceToHost, st));
    // 16-bit stores: the row-staged LB kernel records an expired bulk-copy wait in the controller's third word
    unsigned lb_timeout = 0;
    char* lb_flag = c->ws + c->L.absmax + 2 * sizeof(unsigned);
    if (store_size(c->p) == 2)
        NH_CUDA(c, cudaMemcpyAsync(&lb_timeout, lb_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    NH_CUDA(c, cudaStreamSynchronize(st));
    c->diag_pending = false;
    memset(out, 0, sizeof(*out));
    const double* v = c->host_result;
    out->step = c->step;
    out->mass = v[0] + (c->p.shifted ? (double)(c->has_solid ? c->n_fluid : c->N) : 0.0);
    out->energy = v[1];
    out->max_u = v[2];
    out->min_norm = v[3];
    out->max_norm = v[4];
    out->nonfinite = (int32_t)v[5];
    out->n_tubes = c->diag_tubes;
    const double twopi = 6.283185307179586476925286766559;
    for (int k = 0; k < c->diag_tubes; ++k) {
        const double* t = v + 6 + 5 * k;
        double cx = atan2(t[1], t[2]) * c->p.nx / twopi;
        double cy = atan2(t[3], t[4]) * c->p.ny / twopi;
        if (cx < 0) cx += c->p.nx;
        if (cy < 0) cy += c->p.ny;
        out->centroid[k][0] = cx;
        out->centroid[k][1] = cy;
        out->tube_weight[k] = t[0];
        if (t[0] > 0 && k < c->n_tubes) {
            c->tubes[k][0] = cx;
            c->tubes[k][1] = cy;
            c->tubes_dirty = true;
            c->tubes_epoch += 1;
        }
    }
    if (lb_timeout) {
        NH_CUDA(c, cudaMemsetAsync(lb_flag, 0, sizeof(unsigned), st));
        return fail(c, NH_ETIMEOUT, "a bulk-copy wait of the row-staged LB kernel expired: populations incomplete");
    }
    if (out->nonfinite > 0) return fail(c, NH_EUNSTABLE, "non-finite values in n, u, rho or f");
    return NH_OK;
}

int nh_diagnostics(nh_ctx* c, nh_diag* out)
{
    int r = check_ready(c);
    if (r) return r;
    if (!out) return fail(c, NH_EINVAL, "out is NULL");
    if ((r = nh_diagnostics_enqueue(c, nullptr))) return r;
    return nh_diagnostics_read(c, out);
}

int nh_set_timing(nh_ctx* c, int on)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (on < 0 || on > 2) return fail(c, NH_EINVAL, "timing mode must be 0, 1 or 2");
    close_segment(c);
    c->timing = on;
    return NH_OK;
}

int nh_get_timing(nh_ctx* c, nh_timing* out)
{
    if (!c || !out) return fail(c, NH_EINVAL, "NULL argument");
    close_segment(c);
    if (!c->pending.empty()) {
        for (auto& t : c->pending) {
            cudaError_t e = cudaEventSynchronize(t.b);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, t.a, t.b);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
            c->tstats.launches[t.kclass] += t.count;
            c->tstats.ms[t.kclass] += ms;
            c->free_events.push_back(t.a);
            c->free_events.push_back(t.b);
        }
        c->pending.clear();
    }
    *out = c->tstats;
    memset(&c->tstats, 0, sizeof(c->tstats));
    return NH_OK;
}

int64_t nh_launch_count(const nh_ctx* c) { return c ? c->launches : 0; }

int nh_set_lb_variant(nh_ctx* c, int variant)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (!lb_variant_valid_for(variant, c->p.nx, (int)store_size(c->p)))
        return fail(c, NH_EINVAL, "LB variant not valid for this domain");
    if (variant != c->lb_variant) drop_graphs(c);
    c->lb_variant = variant;
    return NH_OK;
}

int nh_set_diag_fold(nh_ctx* c, int on)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (on != 0 && on != 1) return fail(c, NH_EINVAL, "diag fold must be 0 or 1");
    if (on != c->diag_fold) drop_graphs(c);  // the captured LB launches change
    c->diag_fold = on;
    c->lbp_step = -1;
    c->bdp_step = -1;
    return NH_OK;
}

int nh_set_wait_limit(nh_ctx* c, double seconds)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (isnan(seconds)) return fail(c, NH_EINVAL, "wait limit is NaN");
    c->wait_limit = seconds > 0.0 ? seconds : 0.0;
    return NH_OK;
}

int nh_set_fd_variant(nh_ctx* c, int fused)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    if (fused != 0 && fused != 1) return fail(c, NH_EINVAL, "FD variant must be 0 or 1");
    if (fused && c->p.frank3) return fail(c, NH_EINVAL, "the three-constant energy runs on the per-site FD kernels only");
    if (fused && (c->p.lap_wide || c->p.n_from_rate))
        return fail(c, NH_EINVAL, "lap_wide and n_from_rate run on the per-site FD kernels only");
    if (fused != c->fd_fused) drop_graphs(c);
    c->fd_fused = fused;
    return NH_OK;
}

int nh_autotune(nh_ctx* c, void* stream, int* chosen)
{
    int r = check_ready(c);
    if (r) return r;
    if (!c->fields_set) return fail(c, NH_EINVAL, "nh_set_fields must be called before nh_autotune");
    if ((r = set_device(c))) return r;
    cudaStream_t st = pick(c, stream);
    close_segment(c);
    const int saved_timing = c->timing;
    const int saved_variant = c->lb_variant;
    c->timing = 0;
    cudaEvent_t e0 = get_event(c), e1 = get_event(c);
    float best_ms = 1e30f;
    int best = saved_variant;
    const int reps = 5;
    // Each trial streams the current buffer into the other one without
    // advancing the state (no macro write, no buffer swap).
    for (int v = 0; v < kLBVariantCount && r == NH_OK; ++v) {
        if (!lb_variant_valid_for(v, c->p.nx, (int)store_size(c->p))) continue;
        c->lb_variant = v;
        r = enqueue_lb(c, c->cur, false, st);
        if (r) break;
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && r == NH_OK; ++k) r = enqueue_lb(c, c->cur, false, st);
        cudaEventRecord(e1, st);
        if (r) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) r = cuda_fail(c, e, "cudaEventSynchronize");
        float ms = 0.f;
        if (r == NH_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    c->free_events.push_back(e0);
    c->free_events.push_back(e1);
    c->timing = saved_timing;
    c->lb_variant = best;
    if (best != saved_variant) drop_graphs(c);
    if (chosen) *chosen = best;
    return r;
}

int nh_set_graphs(nh_ctx* c, int on)
{
    if (!c) return fail(nullptr, NH_EINVAL, "ctx is NULL");
    c->use_graphs = on != 0;
    return NH_OK;
}

void nh_destroy(nh_ctx* c)
{
    if (!c) return;
    if (set_device(c) == NH_OK) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        drop_graphs(c);
        close_segment(c);
        for (auto& t : c->pending) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (auto e : c->free_events) cudaEventDestroy(e);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    }
    delete c;
}

}  // extern "C"
