// flic_noalloc.cu — flic_project_noalloc: the spherical projection without any memory
// allocation, for callers that cannot call cudaMalloc (for example code running inside a
// host framework whose device memory is fully owned by its own pool, or a plugin that may
// only touch the buffers it is handed).
//
// The projection needs working memory beyond its inputs and outputs: one 64-bit
// (range, point index) key per pixel, plus the fp32 boundary tables.  Here they live in
// file-scope static device arrays of a fixed maximum size, which every GPU that loads
// libflic holds until the process exits:
//   keys         kNoAllocMaxPixels x 8 B = 2 MiB
//   column table 2 x kNoAllocMaxCols floats, row table 2 x (rows + 1) floats, row order.
// All calls share these arrays and they keep the last call's contents; each call clears
// the keys it uses before projecting.  Calls whose work overlaps on the GPU (two streams,
// two host threads) race on the shared arrays and must be serialised by the caller.
//
// In host code the arrays' names are host-side stand-ins, not device addresses, so their
// device addresses are looked up with cudaGetSymbolAddress on the first call on each
// device (with that device current) and cached.  That first call should therefore come
// before any stream capture.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "flic.h"
#include "flic_internal.h"

constexpr int kNoAllocMaxPixels = FLIC_NOALLOC_MAX_PIXELS;
constexpr int kNoAllocMaxCols = FLIC_NOALLOC_MAX_COLS;
constexpr int kNoAllocMaxRows = FLIC_MAX_ROWS;
constexpr int kMaxDevices = 64;

// the working memory: file-scope static device arrays (see the comment above)
static __device__ __align__(256) unsigned long long g_keys[kNoAllocMaxPixels];
static __device__ __align__(256) float g_colb[2 * kNoAllocMaxCols];
static __device__ __align__(256) float g_rowb[2 * (kNoAllocMaxRows + 1)];
static __device__ __align__(256) int32_t g_srow[kNoAllocMaxRows];

namespace {

struct DevicePtrs {
    bool ready = false;
    unsigned long long* keys = nullptr;
    float* colb = nullptr;
    float* rowb = nullptr;
    int32_t* srow = nullptr;
};

std::mutex g_mu;
DevicePtrs g_dev[kMaxDevices];
// host staging of the tables (fixed size, guarded by g_mu)
float h_colb[2 * kNoAllocMaxCols];
float h_rowb[2 * (kNoAllocMaxRows + 1)];
int32_t h_srow[kNoAllocMaxRows];

flic_status na_fail(flic_status st, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    flic::set_last_error(msg);  // read back with flic_last_error()
    return st;
}

// Projection boundaries (same definition as flic_create's tables): column c starts at
// azimuth c*az_step; row bands are bounded by midpoints of adjacent sorted beam
// elevations, the outer bands half a spacing beyond their beam.  In-place insertion sort,
// no allocation.
bool build_tables(int R, int C, const double* elev, double az_step) {
    if (R < 2) return false;
    for (int c = 0; c < C; ++c) {
        double ang = (double)c * az_step;
        h_colb[2 * c] = (float)std::cos(ang);
        h_colb[2 * c + 1] = (float)std::sin(ang);
    }
    for (int r = 0; r < R; ++r) h_srow[r] = r;
    for (int i = 1; i < R; ++i) {
        int32_t v = h_srow[i];
        int j = i - 1;
        while (j >= 0 && elev[h_srow[j]] > elev[v]) {
            h_srow[j + 1] = h_srow[j];
            --j;
        }
        h_srow[j + 1] = v;
    }
    for (int i = 1; i < R; ++i)
        if (!(elev[h_srow[i]] > elev[h_srow[i - 1]])) return false;
    for (int j = 0; j <= R; ++j) {
        double m;
        if (j == 0) {
            double e0 = elev[h_srow[0]], e1 = elev[h_srow[1]];
            m = e0 - (e1 - e0) / 2.0;
        } else if (j == R) {
            double e0 = elev[h_srow[R - 2]], e1 = elev[h_srow[R - 1]];
            m = e1 + (e1 - e0) / 2.0;
        } else {
            m = (elev[h_srow[j - 1]] + elev[h_srow[j]]) / 2.0;
        }
        h_rowb[2 * j] = (float)std::cos(m);
        h_rowb[2 * j + 1] = (float)std::sin(m);
    }
    return true;
}

flic_status cuda_err(cudaError_t e, const char* what) {
    return na_fail(FLIC_ERR_CUDA, "flic_project_noalloc: %s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" flic_status flic_project_noalloc(int32_t rows, int32_t cols, const double* elevation,
                                            double az_step, const float* xyz, int64_t n,
                                            float* range_out, int32_t* point_pixel,
                                            void* stream) {
    if (rows < 2 || cols < 1 || rows > kNoAllocMaxRows || cols > kNoAllocMaxCols ||
        (int64_t)rows * cols > kNoAllocMaxPixels)
        return na_fail(FLIC_ERR_INVALID,
                       "flic_project_noalloc: %d x %d exceeds the static limits (rows 2..%d, "
                       "cols <= %d, rows*cols <= %d)",
                       rows, cols, kNoAllocMaxRows, kNoAllocMaxCols, kNoAllocMaxPixels);
    if (!elevation || !range_out) return na_fail(FLIC_ERR_INVALID, "flic_project_noalloc: NULL argument");
    if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && (!xyz || !point_pixel)))
        return na_fail(FLIC_ERR_INVALID, "flic_project_noalloc: bad points");
    if (!(az_step > 0.0) || std::fabs((double)cols * az_step - 6.283185307179586) >= 1e-6)
        return na_fail(FLIC_ERR_UNSUPPORTED, "flic_project_noalloc: cols*az_step must be 2 pi");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return na_fail(FLIC_ERR_UNSUPPORTED, "device ordinal too large");
    cudaStream_t s = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lock(g_mu);
    DevicePtrs& d = g_dev[dev];
    if (!d.ready) {
        if ((e = cudaGetSymbolAddress((void**)&d.keys, g_keys)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.colb, g_colb)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.rowb, g_rowb)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.srow, g_srow)) != cudaSuccess)
            return cuda_err(e, "cudaGetSymbolAddress");
        d.ready = true;
    }
    if (!build_tables(rows, cols, elevation, az_step))
        return na_fail(FLIC_ERR_UNSUPPORTED, "flic_project_noalloc: elevations must be distinct");
    // pageable host source: each copy returns once the host data has been staged
    if ((e = cudaMemcpyAsync(d.colb, h_colb, sizeof(float) * 2 * (size_t)cols,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.rowb, h_rowb, sizeof(float) * 2 * (size_t)(rows + 1),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.srow, h_srow, sizeof(int32_t) * (size_t)rows,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_err(e, "table upload");
    flic::ProjDesc P{};
    P.colb = d.colb;
    P.rowb = d.rowb;
    P.srow = d.srow;
    P.rows = rows;
    P.cols = cols;
    P.inv_az_step = (float)(1.0 / az_step);
    P.status = nullptr;
    // launch_project clears the keys of this frame (0xff: empty) before projecting
    if ((e = flic::launch_project(P, xyz, n, d.keys, point_pixel, s)) != cudaSuccess ||
        (e = flic::launch_decode(P, d.keys, range_out, s)) != cudaSuccess)
        return cuda_err(e, "launch");
    return FLIC_OK;
}
