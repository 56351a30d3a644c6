// flic_internal.h — structures shared by the host ABI (flic_api.cu) and the kernels.
// Not part of the public ABI (include/flic.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace flic {

constexpr int kMaxSkip = 8;
constexpr int kMaxCluster = 16;          // thread blocks that cooperate on one work item
constexpr int kMaxStripPixels = 65535;   // local indices (and the run-merge keys) use 16 bits
constexpr int kDefaultIterLimit = 1 << 20;

// One frame as the labelling kernel sees it.  The strip decomposition is part of the
// descriptor: strip s covers columns [s*strip_w, min((s+1)*strip_w, cols)).
struct FrameDesc {
    const float* range;   // rows*cols, device
    int32_t* labels;      // rows*cols, device (output and global union-find forest)
    const float* kv;      // rows*skip, Eq. 3 constants of vertical pairs (upper row)
    const float* kh;      // rows*skip, Eq. 3 constants of horizontal pairs
    int32_t* status;      // device error word of the owning handle
    int32_t rows, cols, skip;
    float delta2;         // delta*delta in fp32
    int32_t wrap;         // 1: column cols-1 neighbours column 0
    int32_t nstrips;      // thread blocks (strips) the frame is split into
    int32_t strip_w;      // columns per strip (last strip may be narrower)
    int32_t pitch_log2;   // local row pitch of the shared-memory forest = 1 << pitch_log2
    int32_t iter_limit;   // bound of every device loop; 0 -> kDefaultIterLimit
    int32_t pad_;
};

// A work item: up to kMaxCluster (frame, strip) pairs processed by one thread-block
// cluster between two cluster barriers.  frame < 0 marks an idle block.
struct ItemDesc {
    int16_t frame[kMaxCluster];
    int16_t strip[kMaxCluster];
};

struct LabelLaunch {
    const FrameDesc* frames;   // device array (batch), or nullptr: use `single`
    const ItemDesc* items;     // device array (batch), or nullptr: one item, rank = strip
    int32_t nitems;
    int32_t cluster;           // blocks per cluster (== blocks per item)
    FrameDesc single;
};

// Shared memory (bytes) one block needs for a strip of `rows` x `width` columns with
// local pitch 1 << pitch_log2 and skip S: the staged readings (rows x (width + S) rounded
// up to 4, later reused as the parent array, rows x pitch ints), the 16-bit edge masks
// (rows x pitch) and two sets of ballot words (rows x pitch / 32 each).
inline size_t strip_smem_bytes(int rows, int pitch_log2, int width, int skip) {
    size_t pitch = size_t(1) << pitch_log2;
    size_t rp = (size_t(width) + size_t(skip) + 3) & ~size_t(3);
    size_t a = size_t(rows) * (rp > pitch ? rp : pitch) * 4;
    size_t mask = size_t(rows) * pitch * 2;
    size_t words = size_t(rows) * (pitch / 32) * 4;  // run ballots + validity ballots
    return a + mask + 2 * words + 64;
}

// Dynamic shared memory one block may use (227 KB opt-in on sm_100/sm_103, minus the
// kernel's static shared memory).
constexpr size_t kMaxDynSmem = 227 * 1024 - 256;

// Kernel launchers (flic_label.cu / flic_project.cu).  Return cudaGetLastError().
cudaError_t launch_label(const LabelLaunch& L, int grid_clusters, int threads, size_t smem,
                         cudaStream_t stream);
cudaError_t launch_edges(const FrameDesc& f, uint16_t* mask, cudaStream_t stream);
cudaError_t label_kernel_setup(size_t max_smem);

struct ProjDesc {
    const float* colb;      // cols x (cos, sin) of the column boundaries
    const float* rowb;      // (rows+1) x (cos, sin) of the sorted elevation boundaries
    const int32_t* srow;    // rows: row index of the j-th lowest beam
    int32_t rows, cols;
    float inv_az_step;      // 1 / az_step, only to seed the column search
    int32_t* status;
};
cudaError_t launch_project(const ProjDesc& P, const float* xyz, int64_t n,
                           unsigned long long* keys, int32_t* point_pixel, cudaStream_t stream);
cudaError_t launch_decode(const ProjDesc& P, const unsigned long long* keys, float* range_out,
                          cudaStream_t stream);
// Sets the thread-local message returned by flic_last_error().
void set_last_error(const char* msg);

cudaError_t launch_scatter(const int32_t* labels, int64_t npix, const int32_t* point_pixel,
                           int64_t n, int32_t* point_labels, cudaStream_t stream);

}  // namespace flic
