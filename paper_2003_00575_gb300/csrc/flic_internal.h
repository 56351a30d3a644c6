// flic_internal.h — structures shared by the host ABI (flic_api.cu) and the kernels.
// Not part of the public ABI (include/flic.h is).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <limits>

#include <cuda_runtime.h>

#include "flic.h"

namespace flic {

constexpr int kMaxSkip = 8;
constexpr int kMaxStrips = 64;           // column strips per frame
constexpr int kMaxStripPixels = 32768;   // rows * pitch of one strip
constexpr int kDefaultIterLimit = 1 << 20;

// One frame as the labelling kernel sees it.  The strip decomposition is part of the
// descriptor: strip s covers columns [s*strip_w, min((s+1)*strip_w, cols)).
struct FrameDesc {
    const float* range;   // rows*cols, device
    int32_t* labels;      // rows*cols, device (output and global union-find forest)
    const float* kv;      // rows*skip, Eq. 3 constants of vertical pairs (upper row)
    const float* kh;      // rows*skip, Eq. 3 constants of horizontal pairs
    const float* kd;      // rows*skip, Eq. 3 constants of diagonal pairs (upper row), or
                          // nullptr when the frame has no diagonal Map Connections
    int32_t* status;      // device error word of the owning handle
    int32_t rows, cols, skip;
    float delta2;         // delta*delta in fp32
    int32_t wrap;         // 1: column cols-1 neighbours column 0
    int32_t nstrips;      // strips the frame is split into
    int32_t strip_w;      // columns per strip (last strip may be narrower)
    int32_t pitch_log2;   // local row pitch of the shared-memory forest = 1 << pitch_log2
    int32_t iter_limit;   // bound of every device loop; 0 -> kDefaultIterLimit
    int32_t lattice;      // 1: offsets 2..skip-1 unused, offset skip only from pixels whose
                          // row and column are multiples of skip (sparse Map Connection)
    // ground extraction (flic_set_ground), nullptr: off.  Row r: [0] sin, [1] cos of the
    // angle to row r-1, [2] tan(gamma - theta), [3] tan(gamma + theta) (gamma = -elevation
    // of row r-1, +-inf past +-90 degrees), [4] sin, [5] cos of row r's elevation.
    const float* gnd;
    float gnd_tan;        // tan(theta), for the height line
    float gnd_height;     // mount height (m); <= 0: no height exception
    // component sizes for flic_label_filter_batch (nullptr: not counted): the size of each
    // component lands at its root's index in cnt, and its root's bit in roots (zero on entry)
    int32_t* cnt;
    uint32_t* roots;
};
constexpr int kGroundFields = 8;  // floats per row of the ground table (6 used)

// One queue entry: P1 (stage, edges, strip-local labels) or P3 (flatten) of one strip.
constexpr int32_t kTaskP1 = 0;
constexpr int32_t kTaskP3 = 1;
struct Task {
    int32_t frame;
    int16_t strip;
    int16_t kind;
};

// Queue counters (int32, zero between launches; the kernel's last block re-zeroes them):
// [kCtrNext] next task, [kCtrExit] blocks done, then kCtrPerFrame per frame f at
// kCtrFrames + kCtrPerFrame*f: [0] borders merged (P3 waits for all), [1] unused,
// [2 + b] strips of border b that finished P1, [kCtrHookRows + s] rows - the topmost row
// of a root of strip s that a border merge hooked (0: none; P3 starts at that row).
constexpr int kCtrNext = 0;
constexpr int kCtrExit = 1;
constexpr int kCtrFrames = 2;
constexpr int kCtrHookRows = 2 + kMaxStrips;
constexpr int kCtrPerFrame = 2 + 2 * kMaxStrips;
static_assert(kCtrHookRows + kMaxStrips <= kCtrPerFrame, "hook rows inside the frame's counters");
__host__ __device__ inline size_t counter_ints(int nframes) {
    return size_t(kCtrFrames) + size_t(kCtrPerFrame) * size_t(nframes);
}

struct LabelLaunch {
    const FrameDesc* frames;   // device array (batch), or nullptr: use `single`
    const Task* tasks;         // device array (batch), or nullptr: implicit single-frame queue
    int32_t ntasks;            // used when dims == nullptr
    int32_t nframes;
    const int32_t* dims;       // device [ntasks, nframes] (batch: uploaded with the tasks)
    int32_t* counters;         // counter_ints(nframes), zero at launch
    FrameDesc single;
};

// Shared memory (bytes) one block needs for a strip of `rows` x `width` columns with
// local pitch 1 << pitch_log2 and skip S: the staged readings (rows x (width + S) rounded
// up to 4, later reused as the parent array, rows x pitch ints) and 2S + 1 ballot words
// per 32-column row segment (twice that with the diagonal Map Connections).
inline size_t strip_smem_bytes(int rows, int pitch_log2, int width, int skip, bool diag = false) {
    size_t pitch = size_t(1) << pitch_log2;
    size_t rp = (size_t(width) + size_t(skip) + 3) & ~size_t(3);
    size_t a = size_t(rows) * (rp > pitch ? rp : pitch) * 4;
    size_t words = size_t(rows) * (pitch / 32) * (2 * size_t(skip) + 1) * 4 * (diag ? 2 : 1);
    return a + words + 64;
}

// Dynamic shared memory one block may use (227 KB opt-in on sm_100/sm_103, minus the
// kernel's static shared memory).
constexpr size_t kMaxDynSmem = 227 * 1024 - 1024;

// Cluster candidates (flic_relabel.cu): per frame, the labels to renumber in place and an
// int32 scratch array of npix (component sizes at root pixels, then their new ids); tiles
// of kRelabelTile pixels, numbered over all frames (frame f's first tile is tile0), each
// with two bitmasks of kRelabelTile bits (roots, kept roots).
constexpr int kRelabelTile = 4096;
constexpr int32_t kRelabelBadLabel = 1;  // == FLIC_ERR_INVALID: a label >= npix was seen
struct RelabelFrame {
    int32_t* labels;
    int32_t* cnt;
    int32_t* num_out;   // device int32: kept components, or nullptr
    int32_t* status;    // the handle's device status word
    int32_t npix;       // <= 2^21
    int32_t tile0;
};
struct RelabelLaunch {
    const RelabelFrame* frames;  // device array, or nullptr: use `single`
    const int32_t* tile_frame;   // device, ntiles: the frame of each tile (nullptr: frame 0)
    int32_t nframes;
    int32_t ntiles;
    int32_t min_size;
    int32_t* tile_cnt;  // ntiles
    int32_t* tile_off;  // ntiles
    uint32_t* roots;    // ntiles x kRelabelTile / 32
    uint32_t* kept;     // ntiles x kRelabelTile / 32
    RelabelFrame single;
};
// Scratch ints a relabel of these frames needs: sizes, two bitmasks, two tile arrays.
inline size_t relabel_scratch_ints(size_t npix_all, size_t ntiles) {
    return npix_all + 2 * ntiles * (kRelabelTile / 32) + 2 * ntiles;
}
// counted: the sizes at the roots and the root bitmask are already there (the labeller
// counted them, FrameDesc::cnt): only count, scan, assign and apply run.
cudaError_t launch_relabel(const RelabelLaunch& L, cudaStream_t stream, bool counted = false);

// Kernel launchers (flic_label.cu / flic_project.cu).  Return cudaGetLastError().
// count: the instance that counts component sizes (frames with FrameDesc::cnt set).
cudaError_t launch_label(const LabelLaunch& L, int grid, int threads, size_t smem,
                         cudaStream_t stream, bool count = false);
cudaError_t label_blocks_per_sm(int threads, size_t smem, int* out);
cudaError_t launch_edges(const FrameDesc& f, uint16_t* mask, cudaStream_t stream);
cudaError_t label_kernel_setup(size_t max_smem);

constexpr int kRowSeeds = 2048;       // buckets of the row-band seed table
constexpr uint32_t kRowOutside = 1023;  // a seed's row field: outside the field of view
// One bucket of the row seed table: t = tan(elevation) of a point below tlo gives row A,
// above thi row B, anything between is settled by the sign tests from band `band`.
struct RowSeed {
    uint32_t info;  // band (bits 0-9) | row A (bits 10-19) | row B (bits 20-29)
    float tlo, thi;
    uint32_t pad;
};
struct ProjDesc {
    const float* colb;      // cols x (cos, sin) of the column boundaries
    const float* rowb;      // (rows+1) x (cos, sin) of the sorted elevation boundaries
    const int32_t* srow;    // rows: row index of the j-th lowest beam
    const RowSeed* rseed;   // kRowSeeds buckets of tan(elevation) between the outer bounds
    float rs_t0, rs_inv_dt; // bucket = (z/rho - rs_t0) * rs_inv_dt; rs_inv_dt 0: no table
    int32_t rows, cols;
    float inv_az_step;      // 1 / az_step, only to seed the column search
    float col_margin;       // a seed's column fraction in (margin, 1 - margin): column holds
    int32_t* status;
};
// The projection's boundary tables, written into caller-supplied arrays (no allocation):
// column c starts at azimuth c*az_step (colb: cols x (cos, sin), fp32 from double); rows are
// sorted by elevation (srow[j] = the row of the j-th lowest beam, a stable insertion sort)
// and bounded by the midpoints of adjacent sorted elevations, the outer bands half a spacing
// beyond their beam (rowb: (rows + 1) x (cos, sin)).  False when rows < 2 or two elevations
// are equal.  flic_create and flic_project_noalloc both build their tables here.
//
// Seeds of the two searches, built so that where they skip the sign tests the tests' answer
// is known.  Both rest on one bound: a boundary more than 1e-6 rad from a point gets the
// sign of the exact test from its fp32 test (whose rounding error is below 4e-7 r).
// - rseed (kRowSeeds buckets of t = tan(elevation) between the outer boundaries): the
//   kernel's bucket of a point (t = z * rsqrt(rho^2), within 2.4e-7 |t| of z / rho) is
//   within one of the point's own, so the point lies in the window of buckets b-1 .. b+1.
//   No boundary within that window (widened by a 1e-6 rad margin): rows A = B = the
//   window's row, limits +inf.  Exactly one boundary k: row A below it (band k-1), row B
//   above (band k), kRowOutside past an outer boundary, and limits T_k -+ m with
//   m = 2e-6 (1 + T_k^2) + 4e-7 (1 + |T_k|), T_k = tan(boundary k), rounded outward: a t
//   outside [tlo, thi] is more than 1e-6 rad from boundary k on the same side.  Two or
//   more: limits -inf, +inf (always settled).  *inv_dt = 0 (no table: a bisection) when an
//   outer boundary lies beyond +-80 degrees.
// - *col_margin: a column seed within 2e-6 rad of the azimuth (the kernel's polynomial is
//   within 1.1e-6) whose column fraction lies in (margin, 1 - margin) keeps both column
//   boundaries more than 1e-6 rad away, counting the fp32 rounding of seed * cols / 2pi.
inline bool build_proj_tables_into(int R, int C, const double* elev, double az_step, float* colb,
                                   float* rowb, int32_t* srow, RowSeed* rseed, float* t0,
                                   float* inv_dt, float* col_margin) {    if (R < 2) return false;
    for (int c = 0; c < C; ++c) {
        const double ang = (double)c * az_step;
        colb[2 * (size_t)c] = (float)std::cos(ang);
        colb[2 * (size_t)c + 1] = (float)std::sin(ang);
    }
    for (int r = 0; r < R; ++r) srow[r] = r;
    for (int i = 1; i < R; ++i) {
        const int32_t v = srow[i];
        int j = i - 1;
        while (j >= 0 && elev[srow[j]] > elev[v]) {
            srow[j + 1] = srow[j];
            --j;
        }
        srow[j + 1] = v;
    }
    for (int i = 1; i < R; ++i)
        if (!(elev[srow[i]] > elev[srow[i - 1]])) return false;
    for (int j = 0; j <= R; ++j) {
        double m;
        if (j == 0) {
            const double e0 = elev[srow[0]], e1 = elev[srow[1]];
            m = e0 - (e1 - e0) / 2.0;
        } else if (j == R) {
            const double e0 = elev[srow[R - 2]], e1 = elev[srow[R - 1]];
            m = e1 + (e1 - e0) / 2.0;
        } else {
            m = (elev[srow[j - 1]] + elev[srow[j]]) / 2.0;
        }
        rowb[2 * (size_t)j] = (float)std::cos(m);
        rowb[2 * (size_t)j + 1] = (float)std::sin(m);
    }
    const double kPi = 3.14159265358979323846;
    *col_margin = (float)(2.0 * C * ((2.0e-6 + 1.0e-6) / (2.0 * kPi) + 1.2e-7));
    if (*col_margin > 0.5f) *col_margin = 0.5f;  // nothing is certain: always settle
    auto bound = [&](int j) {  // boundary j in double, as above
        if (j == 0) return elev[srow[0]] - (elev[srow[1]] - elev[srow[0]]) / 2.0;
        if (j == R) return elev[srow[R - 1]] + (elev[srow[R - 1]] - elev[srow[R - 2]]) / 2.0;
        return (elev[srow[j - 1]] + elev[srow[j]]) / 2.0;
    };
    const double lim = 80.0 * kPi / 180.0;
    const double m0 = bound(0), mR = bound(R);
    *t0 = 0.0f;
    *inv_dt = 0.0f;
    const float inf = std::numeric_limits<float>::infinity();
    for (int b = 0; b < kRowSeeds; ++b) rseed[b] = RowSeed{0u, -inf, inf, 0u};
    if (m0 > -lim && mR < lim && R <= FLIC_MAX_ROWS) {
        double tb[FLIC_MAX_ROWS + 1];  // tan of every boundary, ascending
        for (int j = 0; j <= R; ++j) tb[j] = std::tan(bound(j));
        const double ta = tb[0];
        const double dt = (tb[R] - ta) / kRowSeeds;
        auto row_of = [&](int band) {
            return band < 0 || band >= R ? kRowOutside : (uint32_t)srow[band];
        };
        int j = 0;  // band at the bucket's lower edge
        int k = 0;  // first boundary at or above the window's lower end
        for (int b = 0; b < kRowSeeds; ++b) {
            const double edge = ta + b * dt;
            while (j + 1 < R && tb[j + 1] <= edge) ++j;
            const double wlo = ta + (b - 1) * dt, whi = ta + (b + 2) * dt;
            const double mg = 1.0e-6 * (1.0 + std::max(wlo * wlo, whi * whi));  // 1e-6 rad
            while (k <= R && tb[k] < wlo - mg) ++k;
            int inside = 0;
            while (k + inside <= R && tb[k + inside] <= whi + mg) ++inside;
            RowSeed& e = rseed[b];
            e.info = (uint32_t)j;
            if (inside == 0) {  // the window lies within band j
                e.info |= row_of(j) << 10 | row_of(j) << 20;
                e.tlo = e.thi = inf;
            } else if (inside == 1) {
                const double T = tb[k];
                const double m = 2.0e-6 * (1.0 + T * T) + 4.0e-7 * (1.0 + std::fabs(T));
                e.info |= row_of(k - 1) << 10 | row_of(k) << 20;
                e.tlo = std::nextafter((float)(T - m), -inf);
                e.thi = std::nextafter((float)(T + m), inf);
            }  // else: settled, as initialised
        }
        *t0 = (float)ta;
        *inv_dt = (float)(1.0 / dt);
    }
    return true;
}

cudaError_t launch_project(const ProjDesc& P, const float* xyz, int64_t n,
                           uint32_t* keys, int32_t* point_pixel, cudaStream_t stream);
cudaError_t launch_decode(const ProjDesc& P, const uint32_t* keys, float* range_out,
                          cudaStream_t stream);

// Many clouds projected (and later scattered) by one launch per kernel: every item is one
// cloud with its own handle's tables and key scratch (items passed as kernel parameters).
struct ProjItem {
    ProjDesc P;                   // the handle's tables, shape and status word
    const float* xyz;             // n x 3
    int32_t* point_pixel;         // n
    uint32_t* keys;               // rows x cols, the handle's scratch
    float* range_out;             // rows x cols
    const int32_t* labels;        // rows x cols (scatter)
    int32_t* point_labels;        // n (scatter)
    int32_t n;
};
constexpr int kProjBatchItems = 96;
struct ProjBatch {
    int32_t nitems;
    int32_t max_n;                // largest point count of the items
    int32_t max_px;               // largest pixel count of the items
    ProjItem item[kProjBatchItems];
};
// keys cleared, points projected, range images decoded: three launches for all items
cudaError_t launch_project_batch(const ProjBatch& B, cudaStream_t stream);
// every item's point labels from its pixel labels: one launch
cudaError_t launch_scatter_batch(const ProjBatch& B, cudaStream_t stream);
// Sets the thread-local message returned by flic_last_error().
void set_last_error(const char* msg);

}  // namespace flic
namespace flic {
// A new handle with the same geometry, threshold, skip, flags and tuning as h.
flic_status clone_handle(flic_handle h, flic_handle* out, int* rows, int* cols);
// Launches of batch object b reserve the shared memory of the largest of these frames (with
// b's tuning), so that every mix of them uses one launch shape and one captured graph.
flic_status batch_reserve_smem(flic_batch b, const flic_handle* hs, int n);
// The projection item of one cloud on handle h (FLIC_ERR_UNSUPPORTED when h cannot project).
flic_status proj_item(flic_handle h, const float* xyz, int64_t n, float* range_out,
                      int32_t* point_pixel, const int32_t* labels, int32_t* point_labels,
                      ProjItem* out);

cudaError_t launch_scatter(const int32_t* labels, int64_t npix, const int32_t* point_pixel,
                           int64_t n, int32_t* point_labels, cudaStream_t stream);

}  // namespace flic
