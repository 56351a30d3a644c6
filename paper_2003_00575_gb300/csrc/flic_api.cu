// flic_api.cu — the C ABI of libflic (include/flic.h): handles, host-built tables, the
// strip planner, batch objects with CUDA-graph replay, status reporting.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "flic.h"
#include "flic_internal.h"

namespace {

thread_local std::string g_err;

flic_status fail(flic_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

flic_status cuda_fail(cudaError_t e, const char* what) {
    flic_status st = e == cudaErrorMemoryAllocation ? FLIC_ERR_OOM : FLIC_ERR_CUDA;
    return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kMaxPaddedStrip = flic::kMaxStripPixels;

struct Tuning {
    int px_per_cta = 16384;
    int threads = 512;
    int max_strips = flic::kMaxStrips;
    int ctas_per_sm = 0;  // 0 = as many as fit
    int p3_delay = 8;     // batch: P3 tasks this many waves of blocks after their frame
};

// Strip size of a handle's single-frame calls: one frame alone leaves most SMs idle with
// batch-sized strips, so smaller strips (more blocks per frame) give the lower latency.
constexpr int kSingleFramePx = 2048;

// flic_label_batch_host: groups of frames whose copies overlap the labelling of others
constexpr int kDefaultHostGroups = 4;
constexpr int kMaxHostGroups = 16;

struct StripPlan {
    int nstrips = 0;
    int strip_w = 0;
    int pitch_log2 = 0;
    size_t smem = 0;
};

int ceil_div(int a, int b) { return (a + b - 1) / b; }

int pow2_log2_ceil(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

// Split a rows x cols frame into full-height column strips: about px_target pixels each,
// at most max_strips strips, widths a multiple of 4 (aligned vector access), every strip
// at least `skip` wide when there are several (so an edge crosses at most one border),
// and rows * pitch <= kMaxPaddedStrip with pitch = next power of two >= max(width, 32).
bool plan_frame(int R, int C, int S, int px_target, int max_strips, StripPlan* out,
                bool diag = false) {
    int n0 = std::max(1, std::min(max_strips, ceil_div(std::max(1, R * C), std::max(1, px_target))));
    // preferred strip count first, then more strips, then fewer; for each count a few
    // widths, so that a narrow last strip can be avoided
    std::vector<int> counts;
    for (int n = n0; n <= max_strips; ++n) counts.push_back(n);
    for (int n = n0 - 1; n >= 1; --n) counts.push_back(n);
    for (int n : counts) {
        for (int extra = 0; extra < 4; ++extra) {
            int W = ceil_div(C, n);
            if (n > 1) W = ceil_div(W, 4) * 4 + 4 * extra;
            else if (extra > 0) break;
            int n_eff = ceil_div(C, W);
            if (n_eff > 1) {
                if (W < S) continue;
                int last = C - (n_eff - 1) * W;
                if (last < S) continue;
            }
            int sh = std::max(5, pow2_log2_ceil(W));
            if ((long long)R << sh > kMaxPaddedStrip) continue;
            size_t smem = flic::strip_smem_bytes(R, sh, W, S, diag);
            if (smem > flic::kMaxDynSmem) continue;
            out->nstrips = n_eff;
            out->strip_w = W;
            out->pitch_log2 = sh;
            out->smem = smem;
            return true;
        }
    }
    return false;
}

int device_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Blocks of the label kernel that fit at once (all SMs), capped by ctas_per_sm if set.
int resident_blocks(int threads, size_t smem, int ctas_per_sm) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (flic::label_blocks_per_sm(threads, smem, &per) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    if (ctas_per_sm > 0) per = std::min(per, ctas_per_sm);
    return std::max(1, per) * std::max(1, nsm);
}

}  // namespace

void flic::set_last_error(const char* msg) { g_err = msg; }

struct flic_ctx {
    int R = 0, C = 0, S = 0;
    float delta = 0.0f, delta2 = 0.0f;
    uint32_t flags = 0;
    int wrap = 1;
    double az_step = 0.0;
    int device = 0;
    float* d_kv = nullptr;
    float* d_kh = nullptr;
    float* d_kd = nullptr;  // diagonal Map Connections (FLIC_FLAG_DIAGONAL), else nullptr
    std::vector<float> h_kv, h_kh, h_kd;
    std::vector<double> elev;  // the creation arguments, for flic::clone_handle
    bool proj_ok = false;
    float* d_colb = nullptr;
    float* d_rowb = nullptr;
    int32_t* d_srow = nullptr;
    flic::RowSeed* d_rseed = nullptr;
    float rs_t0 = 0.0f, rs_inv_dt = 0.0f, col_margin = 0.5f;
    float inv_az_step = 0.0f;
    uint32_t* d_keys = nullptr;
    int32_t* d_rl = nullptr;  // flic_filter_relabel scratch (relabel_scratch_ints)
    float* d_gnd = nullptr;   // ground table (flic_set_ground), nullptr: off
    float gnd_tan = 0.0f, gnd_height = 0.0f;
    double gnd_theta_arg = 0.0, gnd_height_arg = 0.0;  // the flic_set_ground arguments
    float* d_range = nullptr;
    int32_t* d_status = nullptr;
    int iter_limit = 0;
    int32_t* d_counters = nullptr;  // task queue of single-frame launches
    int resident = 1;               // blocks of the label kernel that fit at once
    Tuning tune{kSingleFramePx};
    StripPlan plan;
    uint64_t uid = 0;      // unique per handle ever created (pointers can be reused)
    uint64_t version = 0;  // bumped whenever a setting a batch descriptor copies changes
};

struct flic_batch_ctx {
    int max_frames = 0;
    int max_tasks = 0;
    int device = 0;
    size_t min_smem = 0;  // launches reserve at least this much (flic::batch_reserve_smem)
    flic::FrameDesc* h_frames = nullptr;  // pinned staging
    flic::Task* h_tasks = nullptr;
    flic::FrameDesc* d_frames = nullptr;
    flic::Task* d_tasks = nullptr;
    int32_t* d_counters = nullptr;
    int32_t* h_dims = nullptr;  // pinned [ntasks, nframes]
    int32_t* d_dims = nullptr;
    cudaEvent_t staged = nullptr;       // descriptor upload done: staging reusable
    cudaEvent_t kernel_done = nullptr;  // last launch done: device descriptors reusable
    bool pending = false;
    cudaStream_t cap_stream = nullptr;
    Tuning tune;
    std::map<std::tuple<int, int, size_t, bool>, cudaGraphExec_t> graphs;  // grid, threads, smem, counting
    int last_info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // the previous call's arguments and launch shape: an identical call replays the graph
    std::vector<const void*> last_args;
    cudaGraphExec_t last_exec = nullptr;
    // flic_filter_relabel_batch: descriptors (pinned staging + device) and scratch
    flic::RelabelFrame* h_rl = nullptr;
    flic::RelabelFrame* d_rl = nullptr;
    int32_t* d_rl_scratch = nullptr;
    size_t rl_scratch_ints = 0;
    int32_t* h_rl_tile_frame = nullptr;  // pinned: the frame of each tile
    int32_t* d_rl_tile_frame = nullptr;
    size_t rl_tiles = 0;
    cudaEvent_t rl_staged = nullptr;  // descriptor upload done: staging reusable
    cudaEvent_t rl_done = nullptr;    // last relabel done: descriptors and scratch reusable
    bool rl_pending = false;
    // flic_label_batch_host: two sides used by alternate calls, each with device copies of
    // the packed frames, one sub-batch per group of frames (each replays its own graph) and
    // per-group events; copy-in, labelling and copy-out streams
    struct HostSide {
        float* d_range = nullptr;
        int32_t* d_labels = nullptr;
        std::vector<flic_batch_ctx*> subs;
        std::vector<cudaEvent_t> ev_in, ev_lab;
        cudaEvent_t ev_kend = nullptr;  // the side's last labelling done: d_range reusable
        cudaEvent_t ev_dend = nullptr;  // the side's last download done: d_labels reusable
    } side[2];
    size_t host_px_cap = 0;
    uint64_t host_calls = 0;
    cudaStream_t s_in = nullptr, s_lab = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr;
};

namespace {

std::atomic<uint64_t> g_next_uid{1};

flic::FrameDesc frame_desc(const flic_ctx* h, const float* range, int32_t* labels,
                           const StripPlan& pl) {
    flic::FrameDesc f{};
    f.range = range;
    f.labels = labels;
    f.kv = h->d_kv;
    f.kh = h->d_kh;
    f.kd = h->d_kd;
    f.status = h->d_status;
    f.rows = h->R;
    f.cols = h->C;
    f.skip = h->S;
    f.delta2 = h->delta2;
    f.wrap = h->wrap;
    f.nstrips = pl.nstrips;
    f.strip_w = pl.strip_w;
    f.pitch_log2 = pl.pitch_log2;
    f.iter_limit = h->iter_limit;
    f.lattice = (h->flags & FLIC_FLAG_SUBLATTICE) ? 1 : 0;
    f.gnd = h->d_gnd;
    f.gnd_tan = h->gnd_tan;
    f.gnd_height = h->gnd_height;
    return f;
}

// Eq. 3 constants, K = 4 sin^2(alpha/2) = 2 - 2 cos(alpha), in double, rounded once.
void build_k_tables(int R, const double* elev, double az_step, int S, bool exact_ray,
                    std::vector<float>& kv, std::vector<float>& kh) {
    kv.assign((size_t)R * S, 0.0f);
    kh.assign((size_t)R * S, 0.0f);
    for (int r = 0; r < R; ++r) {
        for (int k = 1; k <= S; ++k) {
            float v = 0.0f;
            if (r + k < R) {
                double alpha = std::fabs(elev[r + k] - elev[r]);
                double s = std::sin(alpha / 2.0);
                v = (float)(4.0 * s * s);
            }
            // horizontal: k times the step (§III-B), or the true angle between the two
            // rays of row r: 2 - 2 cos(alpha) = 4 cos^2(e) sin^2(k step / 2)
            double alpha_h = (double)k * az_step;
            double sh = std::sin(alpha_h / 2.0);
            double ce = exact_ray ? std::cos(elev[r]) : 1.0;
            kv[(size_t)r * S + k - 1] = v;
            kh[(size_t)r * S + k - 1] = (float)(4.0 * ce * ce * sh * sh);
        }
    }
}

// Eq. 3 constants of the diagonal pairs (r, c)-(r+k, c+-k): 2 - 2 cos(alpha) with alpha the
// angle between the two rays, as the squared distance |u1 - u2|^2 of the unit rays at
// (elev[r], 0) and (elev[r+k], k * az_step), in double, rounded once (0 where r+k >= R).
std::vector<float> build_kd_table(int R, const double* elev, double az_step, int S) {
    std::vector<float> kd((size_t)R * S, 0.0f);
    for (int r = 0; r < R; ++r)
        for (int k = 1; k <= S && r + k < R; ++k) {
            const double e1 = elev[r], e2 = elev[r + k], ph = (double)k * az_step;
            const double x = std::cos(e1) - std::cos(e2) * std::cos(ph);
            const double y = std::cos(e2) * std::sin(ph);
            const double z = std::sin(e1) - std::sin(e2);
            kd[(size_t)r * S + k - 1] = (float)(x * x + y * y + z * z);
        }
    return kd;
}

// Projection boundaries (flic::build_proj_tables_into) in vectors of the right size.
bool build_proj_tables(int R, int C, const double* elev, double az_step, std::vector<float>& colb,
                       std::vector<float>& rowb, std::vector<int32_t>& srow,
                       std::vector<flic::RowSeed>& rseed, float* t0, float* inv_dt,
                       float* col_margin) {
    if (R < 2) return false;
    colb.resize((size_t)2 * C);
    rowb.resize((size_t)2 * (R + 1));
    srow.resize(R);
    rseed.resize(flic::kRowSeeds);
    return flic::build_proj_tables_into(R, C, elev, az_step, colb.data(), rowb.data(), srow.data(),
                                        rseed.data(), t0, inv_dt, col_margin);
}

template <typename T>
flic_status upload(T** dst, const std::vector<T>& src, const char* what) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(1, src.size()));
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (!src.empty()) {
        e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    return FLIC_OK;
}

void free_ctx(flic_ctx* h) {
    if (!h) return;
    cudaFree(h->d_kv);
    cudaFree(h->d_kh);
    cudaFree(h->d_kd);
    cudaFree(h->d_colb);
    cudaFree(h->d_rowb);
    cudaFree(h->d_srow);
    cudaFree(h->d_rseed);
    cudaFree(h->d_keys);
    cudaFree(h->d_rl);
    cudaFree(h->d_gnd);
    cudaFree(h->d_range);
    cudaFree(h->d_status);
    cudaFree(h->d_counters);
    delete h;
}

flic_status replan(flic_ctx* h) {
    StripPlan pl;
    if (!plan_frame(h->R, h->C, h->S, h->tune.px_per_cta, h->tune.max_strips, &pl,
                    h->d_kd != nullptr))
        return fail(FLIC_ERR_UNSUPPORTED, "frame %dx%d (skip %d) does not fit %d strips",
                    h->R, h->C, h->S, h->tune.max_strips);
    h->plan = pl;
    h->resident = resident_blocks(h->tune.threads, pl.smem, h->tune.ctas_per_sm);
    return FLIC_OK;
}

}  // namespace

extern "C" {

int32_t flic_abi_version(void) { return FLIC_ABI_VERSION; }

const char* flic_last_error(void) { return g_err.c_str(); }

flic_status flic_create(int32_t rows, int32_t cols, const double* elevation, double az_step,
                        float delta, int32_t skip, flic_handle* out) {
    return flic_create_ex(rows, cols, elevation, az_step, delta, skip, 0u, out);
}

flic_status flic_create_ex(int32_t rows, int32_t cols, const double* elevation, double az_step,
                           float delta, int32_t skip, uint32_t flags, flic_handle* out) {
    if (!out) return fail(FLIC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (rows < 1 || cols < 1 || rows > FLIC_MAX_ROWS || (int64_t)rows * cols > FLIC_MAX_PIXELS)
        return fail(FLIC_ERR_INVALID, "bad shape %d x %d (max rows %d, max pixels %d)", rows,
                    cols, FLIC_MAX_ROWS, FLIC_MAX_PIXELS);
    if (!elevation) return fail(FLIC_ERR_INVALID, "elevation is NULL");
    for (int r = 0; r < rows; ++r)
        if (!std::isfinite(elevation[r])) return fail(FLIC_ERR_INVALID, "elevation[%d] not finite", r);
    if (!(az_step > 0.0) || !std::isfinite(az_step))
        return fail(FLIC_ERR_INVALID, "az_step must be positive and finite");
    if (!(delta > 0.0f) || !std::isfinite(delta))
        return fail(FLIC_ERR_INVALID, "delta must be positive and finite");
    if (skip < 1 || skip > FLIC_MAX_SKIP) return fail(FLIC_ERR_INVALID, "skip must be 1..%d", FLIC_MAX_SKIP);
    if (flags & ~(FLIC_FLAG_NO_WRAP | FLIC_FLAG_EXACT_RAY | FLIC_FLAG_SUBLATTICE |
                  FLIC_FLAG_DIAGONAL))
        return fail(FLIC_ERR_INVALID, "unknown flags 0x%x", flags);
    if ((flags & FLIC_FLAG_DIAGONAL) && (flags & FLIC_FLAG_SUBLATTICE))
        return fail(FLIC_ERR_INVALID, "diagonal Map Connections are not combined with the sparse map");

    flic_ctx* h = new flic_ctx();
    h->R = rows;
    h->C = cols;
    h->S = skip;
    h->delta = delta;
    h->delta2 = delta * delta;
    h->flags = flags;
    h->wrap = (flags & FLIC_FLAG_NO_WRAP) ? 0 : 1;
    h->az_step = az_step;
    h->uid = g_next_uid.fetch_add(1);
    h->elev.assign(elevation, elevation + rows);
    cudaGetDevice(&h->device);

    flic_status st;
    cudaError_t e = flic::label_kernel_setup(std::min((size_t)device_max_smem() - 1024, flic::kMaxDynSmem));
    if (e != cudaSuccess) { free_ctx(h); return cuda_fail(e, "kernel attributes"); }

    build_k_tables(rows, elevation, az_step, skip, (flags & FLIC_FLAG_EXACT_RAY) != 0, h->h_kv,
                   h->h_kh);
    if ((st = upload(&h->d_kv, h->h_kv, "Kv table")) != FLIC_OK) { free_ctx(h); return st; }
    if ((st = upload(&h->d_kh, h->h_kh, "Kh table")) != FLIC_OK) { free_ctx(h); return st; }
    if (flags & FLIC_FLAG_DIAGONAL) {
        h->h_kd = build_kd_table(rows, elevation, az_step, skip);
        if ((st = upload(&h->d_kd, h->h_kd, "Kd table")) != FLIC_OK) { free_ctx(h); return st; }
    }
    std::vector<int32_t> zero(1, 0);
    if ((st = upload(&h->d_status, zero, "status word")) != FLIC_OK) { free_ctx(h); return st; }
    std::vector<int32_t> zeros(flic::counter_ints(1), 0);
    if ((st = upload(&h->d_counters, zeros, "task counters")) != FLIC_OK) { free_ctx(h); return st; }

    std::vector<float> colb, rowb;
    std::vector<int32_t> srow;
    std::vector<flic::RowSeed> rseed;
    bool full_turn = std::fabs((double)cols * az_step - kTwoPi) < 1e-6;
    if (full_turn && build_proj_tables(rows, cols, elevation, az_step, colb, rowb, srow, rseed,
                                       &h->rs_t0, &h->rs_inv_dt, &h->col_margin)) {
        if ((st = upload(&h->d_colb, colb, "column boundaries")) != FLIC_OK ||
            (st = upload(&h->d_rowb, rowb, "row boundaries")) != FLIC_OK ||
            (st = upload(&h->d_srow, srow, "row order")) != FLIC_OK ||
            (st = upload(&h->d_rseed, rseed, "row seeds")) != FLIC_OK) {
            free_ctx(h);
            return st;
        }
        size_t npix = (size_t)rows * cols;
        if ((e = cudaMalloc((void**)&h->d_keys, npix * sizeof(uint32_t))) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->d_range, npix * sizeof(float))) != cudaSuccess) {
            free_ctx(h);
            return cuda_fail(e, "projection buffers");
        }
        h->proj_ok = true;
        h->inv_az_step = (float)(1.0 / az_step);
    }
    if ((st = replan(h)) != FLIC_OK) { free_ctx(h); return st; }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { free_ctx(h); return cuda_fail(e, "flic_create"); }
    *out = h;
    return FLIC_OK;
}

flic_status flic_destroy(flic_handle h) {
    if (!h) return FLIC_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_ctx(h);
    if (e != cudaSuccess) return cuda_fail(e, "flic_destroy");
    return FLIC_OK;
}

flic_status flic_get_tables(flic_handle h, float* kv, float* kh) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    if (kv) std::memcpy(kv, h->h_kv.data(), sizeof(float) * h->h_kv.size());
    if (kh) std::memcpy(kh, h->h_kh.data(), sizeof(float) * h->h_kh.size());
    return FLIC_OK;
}

flic_status flic_get_diag_table(flic_handle h, float* kd) {
    if (!h || !kd) return fail(FLIC_ERR_INVALID, "NULL argument");
    if (h->h_kd.empty()) return fail(FLIC_ERR_INVALID, "the handle has no diagonal Map Connections");
    std::memcpy(kd, h->h_kd.data(), sizeof(float) * h->h_kd.size());
    return FLIC_OK;
}

flic_status flic_plan_frame(int32_t rows, int32_t cols, int32_t skip, int32_t px_per_cta,
                            int32_t max_strips, int32_t* info) {
    if (!info || rows < 1 || cols < 1 || skip < 1 || skip > FLIC_MAX_SKIP || px_per_cta < 1 ||
        max_strips < 1 || max_strips > flic::kMaxStrips)
        return fail(FLIC_ERR_INVALID, "bad argument");
    StripPlan pl;
    if (!plan_frame(rows, cols, skip, px_per_cta, max_strips, &pl))
        return fail(FLIC_ERR_UNSUPPORTED, "frame %dx%d does not fit %d strips", rows, cols,
                    max_strips);
    info[0] = pl.nstrips;
    info[1] = pl.strip_w;
    info[2] = 1 << pl.pitch_log2;
    info[3] = (int32_t)pl.smem;
    return FLIC_OK;
}

flic_status flic_plan_info(flic_handle h, int32_t* info) {
    if (!h || !info) return fail(FLIC_ERR_INVALID, "NULL argument");
    info[0] = h->plan.nstrips;
    info[1] = h->plan.strip_w;
    info[2] = 1 << h->plan.pitch_log2;
    info[3] = (int32_t)h->plan.smem;
    info[4] = h->tune.threads;
    return FLIC_OK;
}

flic_status flic_edges(flic_handle h, const float* range, uint16_t* mask, void* stream) {
    if (!h || !range || !mask) return fail(FLIC_ERR_INVALID, "NULL argument");
    flic::FrameDesc f = frame_desc(h, range, nullptr, h->plan);
    cudaError_t e = flic::launch_edges(f, mask, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "flic_edges launch");
    return FLIC_OK;
}

flic_status flic_label(flic_handle h, const float* range, int32_t* labels, void* stream) {
    if (!h || !range || !labels) return fail(FLIC_ERR_INVALID, "NULL argument");
    if ((const void*)range == (const void*)labels) return fail(FLIC_ERR_INVALID, "range aliases labels");
    flic::LabelLaunch L{};
    L.frames = nullptr;
    L.tasks = nullptr;
    L.single = frame_desc(h, range, labels, h->plan);
    const bool border = h->plan.nstrips > 1 || h->wrap;
    L.ntasks = h->plan.nstrips * (border ? 2 : 1);
    L.nframes = 1;
    L.counters = h->d_counters;
    const int grid = std::min(L.ntasks, h->resident);
    cudaError_t e = flic::launch_label(L, grid, h->tune.threads, h->plan.smem, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "flic_label launch");
    return FLIC_OK;
}

flic_status flic_project(flic_handle h, const float* xyz, int64_t n, float* range_out,
                         int32_t* point_pixel, void* stream) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    if (!h->proj_ok)
        return fail(FLIC_ERR_UNSUPPORTED,
                    "projection needs rows >= 2, distinct elevations and cols*az_step = 2 pi");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(FLIC_ERR_INVALID, "bad point count");
    if (n > 0 && (!xyz || !point_pixel)) return fail(FLIC_ERR_INVALID, "NULL argument");
    flic::ProjDesc P{};
    P.colb = h->d_colb;
    P.rowb = h->d_rowb;
    P.srow = h->d_srow;
    P.rseed = h->d_rseed;
    P.rs_t0 = h->rs_t0;
    P.rs_inv_dt = h->rs_inv_dt;
    P.col_margin = h->col_margin;
    P.rows = h->R;
    P.cols = h->C;
    P.inv_az_step = h->inv_az_step;
    P.status = h->d_status;
    float* out = range_out ? range_out : h->d_range;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = flic::launch_project(P, xyz, n, h->d_keys, point_pixel, s);
    if (e == cudaSuccess) e = flic::launch_decode(P, h->d_keys, out, s);
    if (e != cudaSuccess) return cuda_fail(e, "flic_project launch");
    return FLIC_OK;
}

float* flic_range_buffer(flic_handle h) { return h ? h->d_range : nullptr; }

// The clouds' items, in launches of at most kProjBatchItems (a handle's key scratch serves
// one cloud, so a repeated handle is refused).
static flic_status proj_batches(const flic_handle* hs, int32_t nclouds, const float* const* xyz,
                                const int64_t* n, float* const* range_out,
                                int32_t* const* point_pixel, const int32_t* const* labels,
                                int32_t* const* point_labels, std::vector<flic::ProjBatch>& out) {
    if (nclouds < 0) return fail(FLIC_ERR_INVALID, "nclouds < 0");
    if (nclouds > 0 && (!hs || !n || !point_pixel)) return fail(FLIC_ERR_INVALID, "NULL argument");
    std::vector<const flic_ctx*> seen(hs, hs + nclouds);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return fail(FLIC_ERR_INVALID, "a handle appears twice (each cloud needs its own scratch)");
    out.clear();
    for (int i = 0; i < nclouds; ++i) {
        if (!hs[i]) return fail(FLIC_ERR_INVALID, "cloud %d: NULL handle", i);
        if (n[i] > 0 && (!point_pixel[i] || (xyz && !xyz[i]) || (labels && !labels[i]) ||
                         (point_labels && !point_labels[i])))
            return fail(FLIC_ERR_INVALID, "cloud %d: NULL buffer", i);
        if (out.empty() || out.back().nitems == flic::kProjBatchItems) {
            out.emplace_back();
            out.back().nitems = out.back().max_n = out.back().max_px = 0;
        }
        flic::ProjBatch& b = out.back();
        flic::ProjItem& it = b.item[b.nitems];
        flic_status st = flic::proj_item(hs[i], xyz ? xyz[i] : nullptr, n[i],
                                         range_out ? range_out[i] : nullptr, point_pixel[i],
                                         labels ? labels[i] : nullptr,
                                         point_labels ? point_labels[i] : nullptr, &it);
        if (st != FLIC_OK) return st;
        ++b.nitems;
        b.max_n = std::max(b.max_n, it.n);
        b.max_px = std::max(b.max_px, hs[i]->R * hs[i]->C);
    }
    return FLIC_OK;
}

flic_status flic_project_batch(const flic_handle* hs, int32_t nclouds, const float* const* xyz,
                               const int64_t* n, float* const* range_out,
                               int32_t* const* point_pixel, void* stream) {
    if (nclouds > 0 && !xyz) return fail(FLIC_ERR_INVALID, "NULL argument");
    std::vector<flic::ProjBatch> pb;
    flic_status st = proj_batches(hs, nclouds, xyz, n, range_out, point_pixel, nullptr, nullptr, pb);
    if (st != FLIC_OK) return st;
    for (const flic::ProjBatch& b : pb) {
        cudaError_t e = flic::launch_project_batch(b, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "flic_project_batch launch");
    }
    return FLIC_OK;
}

flic_status flic_scatter_batch(const flic_handle* hs, int32_t nclouds, const int32_t* const* labels,
                               const int32_t* const* point_pixel, const int64_t* n,
                               int32_t* const* point_labels, void* stream) {
    if (nclouds > 0 && (!labels || !point_labels)) return fail(FLIC_ERR_INVALID, "NULL argument");
    std::vector<flic::ProjBatch> pb;
    flic_status st = proj_batches(hs, nclouds, nullptr, n, nullptr,
                                  const_cast<int32_t* const*>(point_pixel), labels, point_labels, pb);
    if (st != FLIC_OK) return st;
    for (const flic::ProjBatch& b : pb) {
        cudaError_t e = flic::launch_scatter_batch(b, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "flic_scatter_batch launch");
    }
    return FLIC_OK;
}

flic_status flic_scatter(flic_handle h, const int32_t* labels, const int32_t* point_pixel,
                         int64_t n, int32_t* point_labels, void* stream) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    if (n < 0) return fail(FLIC_ERR_INVALID, "bad point count");
    if (n > 0 && (!labels || !point_pixel || !point_labels))
        return fail(FLIC_ERR_INVALID, "NULL argument");
    cudaError_t e = flic::launch_scatter(labels, (int64_t)h->R * h->C, point_pixel, n,
                                         point_labels, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "flic_scatter launch");
    return FLIC_OK;
}

flic_status flic_set_tuning(flic_handle h, int32_t px_per_cta, int32_t threads, int32_t max_strips) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    if (px_per_cta < 0 || threads < 0 || max_strips < 0 || max_strips > flic::kMaxStrips ||
        (threads && (threads < 128 || threads > 512 || threads % 32)))
        return fail(FLIC_ERR_INVALID, "bad tuning values");
    Tuning old = h->tune;
    Tuning def{kSingleFramePx};
    h->tune.px_per_cta = px_per_cta ? px_per_cta : def.px_per_cta;
    h->tune.threads = threads ? threads : def.threads;
    h->tune.max_strips = max_strips ? max_strips : def.max_strips;
    flic_status st = replan(h);
    if (st != FLIC_OK) {
        h->tune = old;
        replan(h);
    }
    return st;
}

flic_status flic_device_status(flic_handle h, int32_t clear) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "flic_device_status");
    int32_t v = 0;
    e = cudaMemcpy(&v, h->d_status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "flic_device_status read");
    if (clear) {
        int32_t z = 0;
        e = cudaMemcpy(h->d_status, &z, sizeof(z), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemset(h->d_counters, 0, sizeof(int32_t) * flic::counter_ints(1));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();  // landed before any stream's work
        if (e != cudaSuccess) return cuda_fail(e, "flic_device_status clear");
    }
    if (v == flic::kRelabelBadLabel)
        return fail(FLIC_ERR_INVALID, "flic_filter_relabel saw a label outside the frame");
    if (v != 0) return fail(FLIC_ERR_TIMEOUT, "a bounded device loop gave up (status %d)", v);
    return FLIC_OK;
}

flic_status flic_set_ground(flic_handle h, double theta, double mount_height) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    if (!std::isfinite(theta) || !std::isfinite(mount_height) || theta >= 1.5707963267948966)
        return fail(FLIC_ERR_INVALID, "theta must be finite and below 90 degrees");
    cudaError_t e;
    if (!(theta > 0.0) || h->R < 2) {  // off
        if (h->d_gnd) {
            if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "flic_set_ground");
            cudaFree(h->d_gnd);
            h->d_gnd = nullptr;
        }
        h->gnd_tan = h->gnd_height = 0.0f;
        h->gnd_theta_arg = h->gnd_height_arg = 0.0;
        ++h->version;
        return FLIC_OK;
    }
    // per row, in double and rounded once: the constants of Eq. 1's tangent form and the
    // bounds tan(gamma -+ theta) of a horizontal surface, gamma = the upper beam's
    // depression angle
    const double half_pi = 1.5707963267948966;
    std::vector<float> t((size_t)h->R * flic::kGroundFields, 0.0f);
    for (int r = 0; r < h->R; ++r) {
        float* row = t.data() + (size_t)r * flic::kGroundFields;
        row[4] = (float)std::sin(h->elev[r]);
        row[5] = (float)std::cos(h->elev[r]);
        if (r == 0) continue;
        const double alpha = std::fabs(h->elev[r - 1] - h->elev[r]);
        const double gamma = -h->elev[r - 1];
        row[0] = (float)std::sin(alpha);
        row[1] = (float)std::cos(alpha);
        row[2] = gamma - theta <= -half_pi ? -INFINITY : (float)std::tan(gamma - theta);
        row[3] = gamma + theta >= half_pi ? INFINITY : (float)std::tan(gamma + theta);
    }
    if (h->d_gnd) {  // a launch in flight may still read the old table
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "flic_set_ground");
    } else if ((e = cudaMalloc((void**)&h->d_gnd, t.size() * sizeof(float))) != cudaSuccess) {
        return cuda_fail(e, "ground table");
    }
    if ((e = cudaMemcpy(h->d_gnd, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "ground table upload");
    // a copy from pageable memory may return before its DMA lands; work on other
    // (non-blocking) streams must find the table complete
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "ground table upload");
    h->gnd_tan = (float)std::tan(theta);
    h->gnd_height = mount_height > 0.0 ? (float)mount_height : 0.0f;
    h->gnd_theta_arg = theta;
    h->gnd_height_arg = mount_height;
    ++h->version;
    return FLIC_OK;
}

flic_status flic_debug_set_iter_limit(flic_handle h, int32_t limit) {
    if (!h || limit < 0) return fail(FLIC_ERR_INVALID, "bad argument");
    h->iter_limit = limit;
    ++h->version;
    return FLIC_OK;
}

// ------------------------------------------------------------------------------- batch

flic_status flic_batch_create(int32_t max_frames, flic_batch* out) {
    if (!out) return fail(FLIC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (max_frames < 1 || max_frames > (1 << 15))
        return fail(FLIC_ERR_INVALID, "max_frames must be 1..32768");
    flic_batch_ctx* b = new flic_batch_ctx();
    b->max_frames = max_frames;
    b->max_tasks = 2 * flic::kMaxStrips * max_frames;
    cudaGetDevice(&b->device);
    cudaError_t e;
    size_t fb = sizeof(flic::FrameDesc) * (size_t)max_frames;
    size_t tb = sizeof(flic::Task) * (size_t)b->max_tasks;
    size_t cb = sizeof(int32_t) * flic::counter_ints(max_frames);
    if ((e = cudaHostAlloc((void**)&b->h_frames, fb, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&b->h_tasks, tb, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc((void**)&b->d_frames, fb)) != cudaSuccess ||
        (e = cudaMalloc((void**)&b->d_tasks, tb)) != cudaSuccess ||
        (e = cudaMalloc((void**)&b->d_counters, cb)) != cudaSuccess ||
        (e = cudaMemset(b->d_counters, 0, cb)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&b->h_dims, 2 * sizeof(int32_t), cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc((void**)&b->d_dims, 2 * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->kernel_done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&b->h_rl, sizeof(flic::RelabelFrame) * (size_t)max_frames,
                           cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc((void**)&b->d_rl, sizeof(flic::RelabelFrame) * (size_t)max_frames)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->rl_staged, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->rl_done, cudaEventDisableTiming)) != cudaSuccess) {
        flic_batch_destroy(b);
        return cuda_fail(e, "flic_batch_create");
    }
    if ((e = flic::label_kernel_setup(std::min((size_t)device_max_smem() - 1024, flic::kMaxDynSmem))) != cudaSuccess) {
        flic_batch_destroy(b);
        return cuda_fail(e, "kernel attributes");
    }
    *out = b;
    return FLIC_OK;
}

static void clear_graphs(flic_batch_ctx* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->last_args.clear();
    b->last_exec = nullptr;
}

flic_status flic_batch_destroy(flic_batch b) {
    if (!b) return FLIC_OK;
    cudaError_t e = cudaDeviceSynchronize();
    clear_graphs(b);
    if (b->h_frames) cudaFreeHost(b->h_frames);
    if (b->h_tasks) cudaFreeHost(b->h_tasks);
    if (b->h_dims) cudaFreeHost(b->h_dims);
    cudaFree(b->d_dims);
    cudaFree(b->d_frames);
    cudaFree(b->d_tasks);
    cudaFree(b->d_counters);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->kernel_done) cudaEventDestroy(b->kernel_done);
    if (b->h_rl) cudaFreeHost(b->h_rl);
    cudaFree(b->d_rl);
    cudaFree(b->d_rl_scratch);
    cudaFree(b->d_rl_tile_frame);
    if (b->h_rl_tile_frame) cudaFreeHost(b->h_rl_tile_frame);
    if (b->rl_staged) cudaEventDestroy(b->rl_staged);
    if (b->rl_done) cudaEventDestroy(b->rl_done);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (auto& sd : b->side) {
        for (flic_batch_ctx* sub : sd.subs) flic_batch_destroy(sub);
        cudaFree(sd.d_range);
        cudaFree(sd.d_labels);
        for (cudaEvent_t ev : sd.ev_in) cudaEventDestroy(ev);
        for (cudaEvent_t ev : sd.ev_lab) cudaEventDestroy(ev);
        if (sd.ev_kend) cudaEventDestroy(sd.ev_kend);
        if (sd.ev_dend) cudaEventDestroy(sd.ev_dend);
    }
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->s_in) cudaStreamDestroy(b->s_in);
    if (b->s_lab) cudaStreamDestroy(b->s_lab);
    if (b->s_out) cudaStreamDestroy(b->s_out);
    delete b;
    if (e != cudaSuccess) return cuda_fail(e, "flic_batch_destroy");
    return FLIC_OK;
}

flic_status flic_batch_set_tuning(flic_batch b, int32_t px_per_cta, int32_t threads,
                                  int32_t max_strips, int32_t ctas_per_sm) {
    if (!b) return fail(FLIC_ERR_INVALID, "NULL batch");
    if (px_per_cta < 0 || threads < 0 || max_strips < 0 || max_strips > flic::kMaxStrips ||
        ctas_per_sm < 0 || (threads && (threads < 128 || threads > 512 || threads % 32)))
        return fail(FLIC_ERR_INVALID, "bad tuning values");
    if (b->pending) cudaEventSynchronize(b->kernel_done);
    Tuning def;
    b->tune.px_per_cta = px_per_cta ? px_per_cta : def.px_per_cta;
    b->tune.threads = threads ? threads : def.threads;
    b->tune.max_strips = max_strips ? max_strips : def.max_strips;
    b->tune.ctas_per_sm = ctas_per_sm;
    clear_graphs(b);
    return FLIC_OK;
}

flic_status flic_batch_set_schedule(flic_batch b, int32_t p3_delay_waves) {
    if (!b || p3_delay_waves < 0 || p3_delay_waves > 64)
        return fail(FLIC_ERR_INVALID, "p3_delay_waves must be 0..64");
    if (b->pending) cudaEventSynchronize(b->kernel_done);
    b->tune.p3_delay = p3_delay_waves;
    clear_graphs(b);
    return FLIC_OK;
}

flic_status flic_batch_last_plan(flic_batch b, int32_t* info) {
    if (!b || !info) return fail(FLIC_ERR_INVALID, "NULL argument");
    std::memcpy(info, b->last_info, sizeof(b->last_info));
    return FLIC_OK;
}

}  // extern "C"

namespace {

// flic_label_batch, and the labelling step of flic_label_filter_batch: with cnts and roots
// (one each per frame) the kernel also counts the components' sizes (FrameDesc::cnt).
flic_status label_batch_impl(flic_batch b, const flic_handle* hs, const float* const* ranges,
                             int32_t* const* labels, int32_t nframes, void* stream,
                             int32_t* const* cnts, uint32_t* const* roots) {
    if (!b) return fail(FLIC_ERR_INVALID, "NULL batch");
    if (nframes < 0) return fail(FLIC_ERR_INVALID, "nframes < 0");
    if (nframes == 0) return FLIC_OK;
    if (nframes > b->max_frames)
        return fail(FLIC_ERR_BUSY, "%d frames > batch capacity %d", nframes, b->max_frames);
    if (!hs || !ranges || !labels) return fail(FLIC_ERR_INVALID, "NULL argument");
    for (int i = 0; i < nframes; ++i) {
        if (!hs[i] || !ranges[i] || !labels[i])
            return fail(FLIC_ERR_INVALID, "frame %d: NULL handle or buffer", i);
        if ((const void*)ranges[i] == (const void*)labels[i])
            return fail(FLIC_ERR_INVALID, "frame %d: range aliases labels", i);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;

    // identical to the previous call (same handles, buffers, tuning): replay the graph
    std::vector<const void*> args;
    args.reserve((size_t)6 * nframes);
    for (int i = 0; i < nframes; ++i) {
        args.push_back((const void*)(uintptr_t)hs[i]->uid);
        args.push_back((const void*)(uintptr_t)hs[i]->version);
        args.push_back(ranges[i]);
        args.push_back(labels[i]);
        args.push_back(cnts ? cnts[i] : nullptr);
        args.push_back(roots ? roots[i] : nullptr);
    }
    if (b->last_exec && args == b->last_args) {
        // the queue counters are shared with the previous launch: order after it
        e = cudaStreamWaitEvent(st, b->kernel_done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "stream wait");
        e = cudaGraphLaunch(b->last_exec, st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        e = cudaEventRecord(b->kernel_done, st);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
        return FLIC_OK;
    }

    // the pinned staging buffers may still be read by the previous upload
    if (b->pending) {
        e = cudaEventSynchronize(b->staged);
        if (e != cudaSuccess) return cuda_fail(e, "waiting for the previous upload");
    }
    const Tuning& t = b->tune;

    std::vector<StripPlan> plans(nframes);
    size_t smem = 0;
    int total_strips = 0;
    for (int i = 0; i < nframes; ++i) {
        const flic_ctx* h = hs[i];
        if (!plan_frame(h->R, h->C, h->S, t.px_per_cta, t.max_strips, &plans[i], h->d_kd != nullptr))
            return fail(FLIC_ERR_UNSUPPORTED, "frame %d (%dx%d) does not fit %d strips", i, h->R,
                        h->C, t.max_strips);
        smem = std::max(smem, plans[i].smem);
        total_strips += plans[i].nstrips;
        b->h_frames[i] = frame_desc(h, ranges[i], labels[i], plans[i]);
        if (cnts) {
            b->h_frames[i].cnt = cnts[i];
            b->h_frames[i].roots = roots[i];
        }
    }
    smem = std::max(smem, b->min_smem);
    const int resident = resident_blocks(t.threads, smem, t.ctas_per_sm);

    // the queue: P1 tasks of the frames, largest first; P3 tasks of a frame p3_delay waves
    // of blocks after its last P1 task (default 8; one wave is about one P1 task's
    // duration, so with a delay of one a frame's P3 tasks would arrive just as it
    // finishes), so that they seldom wait
    std::vector<int> order(nframes);
    for (int i = 0; i < nframes; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (int64_t)hs[a]->R * hs[a]->C > (int64_t)hs[c]->R * hs[c]->C;
    });
    int nt = 0;
    std::vector<std::pair<int, int>> pending;  // (P1 count after which to emit, frame)
    size_t next_pending = 0;
    auto emit_p3 = [&](int fi) {
        for (int si = 0; si < plans[fi].nstrips; ++si)
            b->h_tasks[nt++] = flic::Task{fi, (int16_t)si, (int16_t)flic::kTaskP3};
    };
    int p1_count = 0;
    for (int oi = 0; oi < nframes; ++oi) {
        const int fi = order[oi];
        for (int si = 0; si < plans[fi].nstrips; ++si) {
            b->h_tasks[nt++] = flic::Task{fi, (int16_t)si, (int16_t)flic::kTaskP1};
            ++p1_count;
            while (next_pending < pending.size() && pending[next_pending].first <= p1_count)
                emit_p3(pending[next_pending++].second);
        }
        const bool border = plans[fi].nstrips > 1 || hs[fi]->wrap;
        if (border) pending.push_back({p1_count + t.p3_delay * resident, fi});
    }
    while (next_pending < pending.size()) emit_p3(pending[next_pending++].second);
    const int ntasks = nt;
    // the whole resident grid every time (idle blocks leave at once), so the captured
    // launch depends only on the block shape and can be replayed for any batch
    const int grid = resident;
    b->h_dims[0] = ntasks;
    b->h_dims[1] = nframes;

    // descriptors: the previous kernel (on whatever stream) must be done reading them
    if (b->pending) {
        e = cudaStreamWaitEvent(st, b->kernel_done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "stream wait");
    }
    e = cudaMemcpyAsync(b->d_frames, b->h_frames, sizeof(flic::FrameDesc) * nframes,
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tasks, b->h_tasks, sizeof(flic::Task) * ntasks,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_dims, b->h_dims, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged, st);
    if (e != cudaSuccess) return cuda_fail(e, "descriptor upload");
    b->pending = true;

    // the persistent kernel, captured once per launch shape and replayed
    auto key = std::make_tuple(grid, t.threads, smem, cnts != nullptr);
    auto found = b->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (found != b->graphs.end()) {
        exec = found->second;
    } else {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
        flic::LabelLaunch L{};
        L.frames = b->d_frames;
        L.tasks = b->d_tasks;
        L.dims = b->d_dims;
        L.counters = b->d_counters;
        cudaError_t le = flic::launch_label(L, grid, t.threads, smem, b->cap_stream,
                                            cnts != nullptr);
        e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le, "batch kernel capture");
        }
        if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        b->graphs[key] = exec;
    }
    e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    e = cudaEventRecord(b->kernel_done, st);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    b->last_args.swap(args);
    b->last_exec = exec;
    int info[8] = {ntasks, grid, t.max_strips, t.threads, (int)smem, total_strips, nframes,
                   resident};
    std::memcpy(b->last_info, info, sizeof(info));
    return FLIC_OK;
}

}  // namespace

extern "C" {

flic_status flic_label_batch(flic_batch b, const flic_handle* hs, const float* const* ranges,
                             int32_t* const* labels, int32_t nframes, void* stream) {
    return label_batch_impl(b, hs, ranges, labels, nframes, stream, nullptr, nullptr);
}

// ------------------------------------------------------------------ batch from host memory

namespace {

bool same_tuning(const Tuning& a, const Tuning& c) {
    return a.px_per_cta == c.px_per_cta && a.threads == c.threads &&
           a.max_strips == c.max_strips && a.ctas_per_sm == c.ctas_per_sm &&
           a.p3_delay == c.p3_delay;
}

// The sub-batch of group g on one side, able to hold n frames, with the parent's launch
// shape.
flic_status host_sub(flic_batch_ctx* b, std::vector<flic_batch_ctx*>& subs, int g, int n,
                     flic_batch_ctx** out) {
    flic_batch_ctx* sub = g < (int)subs.size() ? subs[g] : nullptr;
    if (sub && sub->max_frames < n) {  // too small: replaced (rare; synchronises)
        flic_batch_destroy(sub);
        subs[g] = sub = nullptr;
    }
    if (!sub) {
        flic_status st = flic_batch_create(std::max(n, 1), &sub);
        if (st != FLIC_OK) return st;
        if (g < (int)subs.size()) subs[g] = sub; else subs.push_back(sub);
    }
    if (!same_tuning(sub->tune, b->tune)) {
        if (sub->pending) cudaEventSynchronize(sub->kernel_done);
        sub->tune = b->tune;
        clear_graphs(sub);
    }
    *out = sub;
    return FLIC_OK;
}

cudaError_t make_events(std::vector<cudaEvent_t>& v, int n) {
    while ((int)v.size() < n) {
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        v.push_back(ev);
    }
    return cudaSuccess;
}

}  // namespace

flic_status flic_label_batch_host(flic_batch b, const flic_handle* hs, int32_t nframes,
                                  const float* host_ranges, int32_t* host_labels,
                                  int32_t groups, uint32_t flags, void* stream) {
    if (!b) return fail(FLIC_ERR_INVALID, "NULL batch");
    if (nframes < 0) return fail(FLIC_ERR_INVALID, "nframes < 0");
    if (flags & ~(uint32_t)FLIC_HOST_INPUT_READY) return fail(FLIC_ERR_INVALID, "unknown flags");
    if (nframes == 0) return FLIC_OK;
    if (nframes > b->max_frames)
        return fail(FLIC_ERR_BUSY, "%d frames > batch capacity %d", nframes, b->max_frames);
    if (!hs || !host_ranges || !host_labels) return fail(FLIC_ERR_INVALID, "NULL argument");
    if (groups < 0 || groups > kMaxHostGroups)
        return fail(FLIC_ERR_INVALID, "groups must be 0..%d", kMaxHostGroups);
    std::vector<size_t> off((size_t)nframes + 1, 0);
    for (int i = 0; i < nframes; ++i) {
        if (!hs[i]) return fail(FLIC_ERR_INVALID, "frame %d: NULL handle", i);
        off[i + 1] = off[i] + (size_t)hs[i]->R * hs[i]->C;
    }
    const size_t total = off[nframes];
    {
        const uintptr_t r0 = (uintptr_t)host_ranges, l0 = (uintptr_t)host_labels;
        if (r0 < l0 + 4 * total && l0 < r0 + 4 * total)
            return fail(FLIC_ERR_INVALID, "host ranges overlap host labels");
    }
    // frame-aligned groups of about equal pixel counts, at least one frame each
    const int K = std::min(groups ? groups : kDefaultHostGroups, nframes);
    std::vector<int> first((size_t)K + 1, 0);
    for (int g = 1; g < K; ++g) {
        const size_t target = total * (size_t)g / (size_t)K;
        int j = first[g - 1] + 1;
        while (j < nframes - (K - g) && off[j] < target) ++j;
        first[g] = j;
    }
    first[K] = nframes;

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->s_in) {
        if ((e = cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&b->s_lab, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "flic_label_batch_host streams");
        for (auto& sd : b->side)
            if ((e = cudaEventCreateWithFlags(&sd.ev_kend, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&sd.ev_dend, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "flic_label_batch_host events");
    }
    flic_batch_ctx::HostSide& sd = b->side[b->host_calls & 1];
    if ((e = make_events(sd.ev_in, K)) != cudaSuccess || (e = make_events(sd.ev_lab, K)) != cudaSuccess)
        return cuda_fail(e, "flic_label_batch_host events");
    std::vector<flic_batch_ctx*> sub((size_t)K, nullptr);
    for (int g = 0; g < K; ++g) {
        flic_status s = host_sub(b, sd.subs, g, first[g + 1] - first[g], &sub[g]);
        if (s != FLIC_OK) return s;
    }
    // device copies of the packed frames on both sides (grown after all earlier calls of
    // this kind have finished)
    if (total > b->host_px_cap) {
        if ((e = cudaStreamSynchronize(b->s_out)) != cudaSuccess)
            return cuda_fail(e, "waiting for the previous host batches");
        b->host_px_cap = 0;
        for (auto& side : b->side) {
            cudaFree(side.d_range);
            cudaFree(side.d_labels);
            side.d_range = nullptr;
            side.d_labels = nullptr;
        }
        for (auto& side : b->side)
            if (cudaMalloc((void**)&side.d_range, 4 * total) != cudaSuccess ||
                cudaMalloc((void**)&side.d_labels, 4 * total) != cudaSuccess) {
                cudaGetLastError();
                return fail(FLIC_ERR_OOM, "device copies of %zu pixels", total);
            }
        b->host_px_cap = total;
    }

    // this side's buffers: the uploads follow its previous labelling, the labelling its
    // previous download; without FLIC_HOST_INPUT_READY both also follow `stream`
    if ((e = cudaStreamWaitEvent(b->s_in, sd.ev_kend, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->s_lab, sd.ev_dend, 0)) != cudaSuccess)
        return cuda_fail(e, "stream ordering");
    if (!(flags & FLIC_HOST_INPUT_READY) &&
        ((e = cudaEventRecord(b->ev_start, st)) != cudaSuccess ||
         (e = cudaStreamWaitEvent(b->s_in, b->ev_start, 0)) != cudaSuccess ||
         (e = cudaStreamWaitEvent(b->s_lab, b->ev_start, 0)) != cudaSuccess))
        return cuda_fail(e, "stream ordering");
    // all uploads first, so that the copy stream never waits on the host
    for (int g = 0; g < K; ++g) {
        const size_t p0 = off[first[g]], n = off[first[g + 1]] - p0;
        if ((e = cudaMemcpyAsync(sd.d_range + p0, host_ranges + p0, 4 * n,
                                 cudaMemcpyHostToDevice, b->s_in)) != cudaSuccess ||
            (e = cudaEventRecord(sd.ev_in[g], b->s_in)) != cudaSuccess)
            return cuda_fail(e, "range upload");
    }
    std::vector<const float*> rp;
    std::vector<int32_t*> lp;
    for (int g = 0; g < K; ++g) {
        const int f0 = first[g], nf = first[g + 1] - f0;
        rp.resize(nf);
        lp.resize(nf);
        for (int i = 0; i < nf; ++i) {
            rp[i] = sd.d_range + off[f0 + i];
            lp[i] = sd.d_labels + off[f0 + i];
        }
        if ((e = cudaStreamWaitEvent(b->s_lab, sd.ev_in[g], 0)) != cudaSuccess)
            return cuda_fail(e, "stream ordering");
        flic_status s = flic_label_batch(sub[g], hs + f0, rp.data(), lp.data(), nf, b->s_lab);
        if (s != FLIC_OK) return s;
        const size_t p0 = off[f0], n = off[first[g + 1]] - p0;
        if ((e = cudaEventRecord(sd.ev_lab[g], b->s_lab)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(b->s_out, sd.ev_lab[g], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(host_labels + p0, sd.d_labels + p0, 4 * n,
                                 cudaMemcpyDeviceToHost, b->s_out)) != cudaSuccess)
            return cuda_fail(e, "label download");
    }
    if ((e = cudaEventRecord(sd.ev_kend, b->s_lab)) != cudaSuccess ||
        (e = cudaEventRecord(sd.ev_dend, b->s_out)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, sd.ev_dend, 0)) != cudaSuccess)
        return cuda_fail(e, "stream ordering");
    ++b->host_calls;
    return FLIC_OK;
}

namespace {

// Carve a relabel scratch block: sizes (npix_all), root and kept bitmasks, tile arrays.
void carve_relabel(flic::RelabelLaunch* L, int32_t* base, size_t npix_all, int ntiles) {
    L->roots = reinterpret_cast<uint32_t*>(base + npix_all);
    L->kept = L->roots + (size_t)ntiles * (flic::kRelabelTile / 32);
    L->tile_cnt = reinterpret_cast<int32_t*>(L->kept + (size_t)ntiles * (flic::kRelabelTile / 32));
    L->tile_off = L->tile_cnt + ntiles;
}

}  // namespace

flic_status flic_filter_relabel(flic_handle h, int32_t* labels, int32_t min_size,
                                int32_t* num_out, void* stream) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    if (!labels) return fail(FLIC_ERR_INVALID, "NULL labels");
    const int npix = h->R * h->C;
    const int ntiles = (npix + flic::kRelabelTile - 1) / flic::kRelabelTile;
    cudaError_t e;
    if (!h->d_rl) {
        const size_t ints = flic::relabel_scratch_ints((size_t)npix, (size_t)ntiles);
        if ((e = cudaMalloc((void**)&h->d_rl, ints * sizeof(int32_t))) != cudaSuccess)
            return cuda_fail(e, "relabel scratch");
    }
    flic::RelabelLaunch L{};
    L.nframes = 1;
    L.ntiles = ntiles;
    L.min_size = min_size;
    carve_relabel(&L, h->d_rl, (size_t)npix, ntiles);
    L.single = {labels, h->d_rl, num_out, h->d_status, npix, 0};
    e = flic::launch_relabel(L, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "flic_filter_relabel launch");
    return FLIC_OK;
}

}  // extern "C"

namespace {

// The relabel launch of nframes frames: scratch (grown when needed), per-frame descriptors
// and the tile map, uploaded on the stream after the previous relabel of this batch.
flic_status relabel_prepare(flic_batch b, const flic_handle* hs, int32_t* const* labels,
                            int32_t nframes, int32_t min_size, int32_t* num_out,
                            cudaStream_t st, flic::RelabelLaunch* out) {
    cudaError_t e;
    size_t npix_all = 0;
    int ntiles = 0;
    for (int i = 0; i < nframes; ++i) {
        if (!hs[i] || !labels[i]) return fail(FLIC_ERR_INVALID, "NULL handle or labels %d", i);
        const int npix = hs[i]->R * hs[i]->C;
        npix_all += (size_t)npix;
        ntiles += (npix + flic::kRelabelTile - 1) / flic::kRelabelTile;
    }
    // the pinned staging may still be read by the previous upload, the scratch and the
    // device descriptors by the previous launches
    if (b->rl_pending && (e = cudaEventSynchronize(b->rl_staged)) != cudaSuccess)
        return cuda_fail(e, "waiting for the previous upload");
    const size_t need = flic::relabel_scratch_ints(npix_all, (size_t)ntiles);
    if (need > b->rl_scratch_ints || (size_t)ntiles > b->rl_tiles) {
        if (b->rl_pending && (e = cudaEventSynchronize(b->rl_done)) != cudaSuccess)
            return cuda_fail(e, "waiting for the previous relabel");
        cudaFree(b->d_rl_scratch);
        cudaFree(b->d_rl_tile_frame);
        cudaFreeHost(b->h_rl_tile_frame);
        b->d_rl_scratch = nullptr;
        b->d_rl_tile_frame = b->h_rl_tile_frame = nullptr;
        b->rl_scratch_ints = b->rl_tiles = 0;
        if ((e = cudaMalloc((void**)&b->d_rl_scratch, need * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc((void**)&b->d_rl_tile_frame, ntiles * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaHostAlloc((void**)&b->h_rl_tile_frame, ntiles * sizeof(int32_t),
                               cudaHostAllocDefault)) != cudaSuccess)
            return cuda_fail(e, "relabel scratch");
        b->rl_scratch_ints = need;
        b->rl_tiles = (size_t)ntiles;
    }
    int tile0 = 0;
    size_t off = 0;
    for (int i = 0; i < nframes; ++i) {
        const int npix = hs[i]->R * hs[i]->C;
        const int nt = (npix + flic::kRelabelTile - 1) / flic::kRelabelTile;
        b->h_rl[i] = {labels[i], b->d_rl_scratch + off, num_out ? num_out + i : nullptr,
                      hs[i]->d_status, npix, tile0};
        for (int k = 0; k < nt; ++k) b->h_rl_tile_frame[tile0 + k] = i;
        off += (size_t)npix;
        tile0 += nt;
    }
    if (b->rl_pending && (e = cudaStreamWaitEvent(st, b->rl_done, 0)) != cudaSuccess)
        return cuda_fail(e, "stream wait");
    e = cudaMemcpyAsync(b->d_rl, b->h_rl, sizeof(flic::RelabelFrame) * nframes,
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_rl_tile_frame, b->h_rl_tile_frame, sizeof(int32_t) * ntiles,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->rl_staged, st);
    if (e != cudaSuccess) return cuda_fail(e, "descriptor upload");
    b->rl_pending = true;
    flic::RelabelLaunch L{};
    L.frames = b->d_rl;
    L.tile_frame = b->d_rl_tile_frame;
    L.nframes = nframes;
    L.ntiles = ntiles;
    L.min_size = min_size;
    carve_relabel(&L, b->d_rl_scratch, npix_all, ntiles);
    *out = L;
    return FLIC_OK;
}

}  // namespace

extern "C" {

flic_status flic_filter_relabel_batch(flic_batch b, const flic_handle* hs,
                                      int32_t* const* labels, int32_t nframes, int32_t min_size,
                                      int32_t* num_out, void* stream) {
    if (!b || !hs || !labels) return fail(FLIC_ERR_INVALID, "NULL argument");
    if (nframes < 0 || nframes > b->max_frames)
        return fail(FLIC_ERR_INVALID, "nframes must be 0..%d", b->max_frames);
    if (nframes == 0) return FLIC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    flic::RelabelLaunch L{};
    flic_status fs = relabel_prepare(b, hs, labels, nframes, min_size, num_out, st, &L);
    if (fs != FLIC_OK) return fs;
    cudaError_t e = flic::launch_relabel(L, st);
    if (e != cudaSuccess) return cuda_fail(e, "flic_filter_relabel_batch launch");
    if ((e = cudaEventRecord(b->rl_done, st)) != cudaSuccess) return cuda_fail(e, "event record");
    return FLIC_OK;
}

flic_status flic_label_filter_batch(flic_batch b, const flic_handle* hs,
                                    const float* const* ranges, int32_t* const* labels,
                                    int32_t nframes, int32_t min_size, int32_t* num_out,
                                    void* stream) {
    if (!b || !hs || !ranges || !labels) return fail(FLIC_ERR_INVALID, "NULL argument");
    if (nframes < 0 || nframes > b->max_frames)
        return fail(FLIC_ERR_INVALID, "nframes must be 0..%d", b->max_frames);
    if (nframes == 0) return FLIC_OK;
    for (int i = 0; i < nframes; ++i)
        if (!hs[i] || !ranges[i] || !labels[i])
            return fail(FLIC_ERR_INVALID, "frame %d: NULL handle or buffer", i);
    cudaStream_t st = (cudaStream_t)stream;
    flic::RelabelLaunch L{};
    flic_status fs = relabel_prepare(b, hs, labels, nframes, min_size, num_out, st, &L);
    if (fs != FLIC_OK) return fs;
    // the root bitmask is built by the labeller's atomics: zero it first (the scratch is
    // the relabel's, ordered after the previous relabel by relabel_prepare)
    cudaError_t e = cudaMemsetAsync(L.roots, 0,
                                    (size_t)L.ntiles * (flic::kRelabelTile / 32) * sizeof(uint32_t),
                                    st);
    if (e != cudaSuccess) return cuda_fail(e, "root bitmask clear");
    std::vector<int32_t*> cnts(nframes);
    std::vector<uint32_t*> roots(nframes);
    for (int i = 0; i < nframes; ++i) {
        cnts[i] = b->h_rl[i].cnt;
        roots[i] = L.roots + (size_t)b->h_rl[i].tile0 * (flic::kRelabelTile / 32);
    }
    fs = label_batch_impl(b, hs, ranges, labels, nframes, stream, cnts.data(), roots.data());
    if (fs != FLIC_OK) return fs;
    e = flic::launch_relabel(L, st, /*counted=*/true);
    if (e != cudaSuccess) return cuda_fail(e, "flic_label_filter_batch relabel launch");
    if ((e = cudaEventRecord(b->rl_done, st)) != cudaSuccess) return cuda_fail(e, "event record");
    return FLIC_OK;
}

}  // extern "C"

flic_status flic::batch_reserve_smem(flic_batch b, const flic_handle* hs, int n) {
    if (!b || (n > 0 && !hs)) return fail(FLIC_ERR_INVALID, "NULL argument");
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        StripPlan pl;
        if (!hs[i] || !plan_frame(hs[i]->R, hs[i]->C, hs[i]->S, b->tune.px_per_cta,
                                  b->tune.max_strips, &pl, hs[i]->d_kd != nullptr))
            return fail(FLIC_ERR_UNSUPPORTED, "frame %d does not fit the batch's strips", i);
        smem = std::max(smem, pl.smem);
    }
    if (b->pending) cudaEventSynchronize(b->kernel_done);
    b->min_smem = smem;
    clear_graphs(b);
    return FLIC_OK;
}

flic_status flic::proj_item(flic_handle h, const float* xyz, int64_t n, float* range_out,
                            int32_t* point_pixel, const int32_t* labels, int32_t* point_labels,
                            flic::ProjItem* out) {
    if (!h || !out) return fail(FLIC_ERR_INVALID, "NULL argument");
    if (!h->proj_ok)
        return fail(FLIC_ERR_UNSUPPORTED,
                    "projection needs rows >= 2, distinct elevations and cols*az_step = 2 pi");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(FLIC_ERR_INVALID, "bad point count");
    flic::ProjItem it{};
    it.P.colb = h->d_colb;
    it.P.rowb = h->d_rowb;
    it.P.srow = h->d_srow;
    it.P.rseed = h->d_rseed;
    it.P.rs_t0 = h->rs_t0;
    it.P.rs_inv_dt = h->rs_inv_dt;
    it.P.col_margin = h->col_margin;
    it.P.rows = h->R;
    it.P.cols = h->C;
    it.P.inv_az_step = h->inv_az_step;
    it.P.status = h->d_status;
    it.xyz = xyz;
    it.point_pixel = point_pixel;
    it.keys = h->d_keys;
    it.range_out = range_out ? range_out : h->d_range;
    it.labels = labels;
    it.point_labels = point_labels;
    it.n = (int32_t)n;
    *out = it;
    return FLIC_OK;
}

flic_status flic::clone_handle(flic_handle h, flic_handle* out, int* rows, int* cols) {
    if (!h) return fail(FLIC_ERR_INVALID, "NULL handle");
    *rows = h->R;
    *cols = h->C;
    flic_status st = flic_create_ex(h->R, h->C, h->elev.data(), h->az_step, h->delta, h->S,
                                    h->flags, out);
    if (st == FLIC_OK) {
        (*out)->tune = h->tune;
        replan(*out);
        if (h->d_gnd) st = flic_set_ground(*out, h->gnd_theta_arg, h->gnd_height_arg);
    }
    return st;
}
