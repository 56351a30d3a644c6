// flic_noalloc.cu — flic_project_noalloc: the spherical projection without any memory
// allocation, for callers that cannot call cudaMalloc (for example code running inside a
// host framework whose device memory is fully owned by its own pool, or a plugin that may
// only touch the buffers it is handed).
//
// The projection needs working memory beyond its inputs and outputs: one 64-bit
// (range, point index) key per pixel, plus the fp32 boundary tables and a status word.
// Here they live in file-scope static device arrays of a fixed maximum size, which every
// GPU that loads libflic holds until the process exits:
//   keys         kNoAllocMaxPixels x 8 B = 2 MiB
//   column table 2 x kNoAllocMaxCols floats, row table 2 x (rows + 1) floats, row order,
//   status       one int32 (a bounded search that gave up)
// All calls share these arrays and they keep the last call's contents; each call clears
// the keys it uses and the status word before projecting.  Calls whose work overlaps on
// the GPU (two streams, two host threads) race on the shared arrays and must be
// serialised by the caller.
//
// In host code the arrays' names are host-side stand-ins, not device addresses, so their
// device addresses are looked up with cudaGetSymbolAddress on the first call on each
// device (with that device current) and cached.
//
// The tables are uploaded from fixed host arrays that every call overwrites, so the call
// cannot be captured into a CUDA graph (a replay would read whatever those arrays hold
// then): it refuses a capturing stream.  It also waits for its own work at the end, which
// lets it report a bounded search that gave up as FLIC_ERR_TIMEOUT.
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
static __device__ __align__(256) uint32_t g_keys[kNoAllocMaxPixels];
static __device__ __align__(256) float g_colb[2 * kNoAllocMaxCols];
static __device__ __align__(256) float g_rowb[2 * (kNoAllocMaxRows + 1)];
static __device__ __align__(256) int32_t g_srow[kNoAllocMaxRows];
static __device__ __align__(256) flic::RowSeed g_rseed[flic::kRowSeeds];
static __device__ __align__(256) int32_t g_status;

namespace {

struct DevicePtrs {
    bool ready = false;
    uint32_t* keys = nullptr;
    float* colb = nullptr;
    float* rowb = nullptr;
    int32_t* srow = nullptr;
    flic::RowSeed* rseed = nullptr;
    int32_t* status = nullptr;
};

std::mutex g_mu;
DevicePtrs g_dev[kMaxDevices];
// host staging of the tables (fixed size, guarded by g_mu)
float h_colb[2 * kNoAllocMaxCols];
float h_rowb[2 * (kNoAllocMaxRows + 1)];
int32_t h_srow[kNoAllocMaxRows];
flic::RowSeed h_rseed[flic::kRowSeeds];

flic_status na_fail(flic_status st, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    flic::set_last_error(msg);  // read back with flic_last_error()
    return st;
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
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return cuda_err(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return na_fail(FLIC_ERR_UNSUPPORTED,
                       "flic_project_noalloc cannot be captured: its tables come from host "
                       "arrays that later calls overwrite");

    std::lock_guard<std::mutex> lock(g_mu);
    DevicePtrs& d = g_dev[dev];
    if (!d.ready) {
        if ((e = cudaGetSymbolAddress((void**)&d.keys, g_keys)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.colb, g_colb)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.rowb, g_rowb)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.srow, g_srow)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.rseed, g_rseed)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&d.status, g_status)) != cudaSuccess)
            return cuda_err(e, "cudaGetSymbolAddress");
        d.ready = true;
    }
    float rs_t0 = 0.0f, rs_inv_dt = 0.0f, col_margin = 0.5f;
    if (!flic::build_proj_tables_into(rows, cols, elevation, az_step, h_colb, h_rowb, h_srow,
                                      h_rseed, &rs_t0, &rs_inv_dt, &col_margin))
        return na_fail(FLIC_ERR_UNSUPPORTED, "flic_project_noalloc: elevations must be distinct");
    // pageable host source: each copy returns once the host data has been staged
    if ((e = cudaMemcpyAsync(d.colb, h_colb, sizeof(float) * 2 * (size_t)cols,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.rowb, h_rowb, sizeof(float) * 2 * (size_t)(rows + 1),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.srow, h_srow, sizeof(int32_t) * (size_t)rows,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d.rseed, h_rseed, sizeof(h_rseed), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(d.status, 0, sizeof(int32_t), s)) != cudaSuccess)
        return cuda_err(e, "table upload");
    flic::ProjDesc P{};
    P.colb = d.colb;
    P.rowb = d.rowb;
    P.srow = d.srow;
    P.rseed = d.rseed;
    P.rs_t0 = rs_t0;
    P.rs_inv_dt = rs_inv_dt;
    P.col_margin = col_margin;
    P.rows = rows;
    P.cols = cols;
    P.inv_az_step = (float)(1.0 / az_step);
    P.status = d.status;
    // launch_project clears the keys of this frame (0xff: empty) before projecting
    if ((e = flic::launch_project(P, xyz, n, d.keys, point_pixel, s)) != cudaSuccess ||
        (e = flic::launch_decode(P, d.keys, range_out, s)) != cudaSuccess)
        return cuda_err(e, "launch");
    int32_t st = 0;
    if ((e = cudaMemcpyAsync(&st, d.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_err(e, "completion");
    if (st != 0)
        return na_fail(FLIC_ERR_TIMEOUT,
                       "flic_project_noalloc: a bounded pixel search gave up; the pixel map is "
                       "not valid");
    return FLIC_OK;
}
