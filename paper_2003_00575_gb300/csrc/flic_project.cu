// flic_project.cu — spherical projection of an xyz cloud into the range image and the
// scatter of pixel labels back onto the points (§I, Fig. 1; §IV-B on one-to-one
// point/pixel matching).
//
// Bin membership is decided only by exact fp32 sign tests against boundary vectors built
// on the host in double and rounded once:
//   column c  iff  cos(c d)*y - sin(c d)*x >= 0  and  cos((c+1) d)*y - sin((c+1) d)*x < 0
//   row band j (sorted boundaries m_j < m_j+1)  iff  cos(m_j)*z - sin(m_j)*rho >= 0 and
//                                                    cos(m_j+1)*z - sin(m_j+1)*rho < 0
// atan2f only seeds the column search; the answer never depends on its rounding.
// Each product, sum and square root is a separately rounded fp32 operation.
// A pixel keeps the point with the smallest range, ties to the lower point index: one
// 64-bit atomicMin on (range bits << 32 | index), positive floats ordering like their bits.
#include <cstdint>

#include "flic_device.cuh"
#include "flic_internal.h"

namespace flic {

namespace {

constexpr float kTwoPiF = 6.28318530717958647692f;

__device__ __forceinline__ float s_col(const float* __restrict__ colb, int C, int c, float x,
                                       float y) {
    const int i = c >= C ? c - C : c;
    return __fsub_rn(__fmul_rn(__ldg(colb + 2 * i), y), __fmul_rn(__ldg(colb + 2 * i + 1), x));
}

__device__ __forceinline__ float s_row(const float* __restrict__ rowb, int j, float z,
                                       float rho) {
    return __fsub_rn(__fmul_rn(__ldg(rowb + 2 * j), z), __fmul_rn(__ldg(rowb + 2 * j + 1), rho));
}

// Point i of a cloud: its pixel (or -1), and its key offered to the pixel.
__device__ __forceinline__ int32_t project_point(const ProjDesc& P, const float* __restrict__ xyz,
                                                 int64_t i, unsigned long long* __restrict__ keys) {
    const float x = __ldg(xyz + 3 * i);
    const float y = __ldg(xyz + 3 * i + 1);
    const float z = __ldg(xyz + 3 * i + 2);
    const float rho2 = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
    const float r2 = __fadd_rn(rho2, __fmul_rn(z, z));
    const float rho = __fsqrt_rn(rho2);
    const float rg = __fsqrt_rn(r2);
    int32_t pix = -1;
    if (valid_range(rg) && rho > 0.0f && s_row(P.rowb, 0, z, rho) >= 0.0f &&
        s_row(P.rowb, P.rows, z, rho) < 0.0f) {
        // row band by bisection: s(lo) >= 0, s(hi) < 0
        int lo = 0, hi = P.rows;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_row(P.rowb, mid, z, rho) >= 0.0f) lo = mid; else hi = mid;
        }
        // column: seeded by atan2f, settled by the sign tests
        float phi = atan2f(y, x);
        if (phi < 0.0f) phi += kTwoPiF;
        int c = (int)floorf(phi * P.inv_az_step);
        c = c < 0 ? 0 : (c >= P.cols ? P.cols - 1 : c);
        bool settled = false;
        for (int it = 0; it < 64; ++it) {
            if (s_col(P.colb, P.cols, c + 1, x, y) >= 0.0f) {
                c = c + 1 == P.cols ? 0 : c + 1;
            } else if (s_col(P.colb, P.cols, c, x, y) < 0.0f) {
                c = c == 0 ? P.cols - 1 : c - 1;
            } else {
                settled = true;
                break;
            }
        }
        if (!settled) report_timeout(P.status);
        pix = __ldg(P.srow + lo) * P.cols + c;
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(rg) << 32) | (unsigned long long)(uint32_t)i;
        atomicMin(keys + pix, key);
    }
    return pix;
}

__global__ void flic_project_kernel(const ProjDesc P, const float* __restrict__ xyz, int64_t n,
                                    unsigned long long* __restrict__ keys,
                                    int32_t* __restrict__ point_pixel) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        point_pixel[i] = project_point(P, xyz, i, keys);
}

// ---- many clouds per launch: blockIdx.y is the item, x strides over its points or pixels

__global__ void flic_clear_keys_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    const int npix = it.P.rows * it.P.cols;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x)
        it.keys[p] = ~0ull;
}

__global__ void flic_project_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < it.n; i += gridDim.x * blockDim.x)
        it.point_pixel[i] = project_point(it.P, it.xyz, i, it.keys);
}

__global__ void flic_decode_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    const int npix = it.P.rows * it.P.cols;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const unsigned long long k = it.keys[p];
        it.range_out[p] = k == ~0ull ? 0.0f : __uint_as_float((unsigned)(k >> 32));
    }
}

__global__ void flic_scatter_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    const int npix = it.P.rows * it.P.cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < it.n; i += gridDim.x * blockDim.x) {
        const int32_t p = __ldg(it.point_pixel + i);
        it.point_labels[i] = (p >= 0 && p < npix) ? __ldg(it.labels + p) : -1;
    }
}

__global__ void flic_decode_kernel(const unsigned long long* __restrict__ keys, int npix,
                                   float* __restrict__ range_out) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[p];
        range_out[p] = k == ~0ull ? 0.0f : __uint_as_float((unsigned)(k >> 32));
    }
}

__global__ void flic_scatter_kernel(const int32_t* __restrict__ labels, int64_t npix,
                                    const int32_t* __restrict__ point_pixel, int64_t n,
                                    int32_t* __restrict__ point_labels) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t p = __ldg(point_pixel + i);
        point_labels[i] = (p >= 0 && p < npix) ? __ldg(labels + p) : -1;
    }
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

cudaError_t launch_project(const ProjDesc& P, const float* xyz, int64_t n,
                           unsigned long long* keys, int32_t* point_pixel, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * (size_t)P.rows *
                                                    (size_t)P.cols, stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        flic_project_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(P, xyz, n, keys, point_pixel);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode(const ProjDesc& P, const unsigned long long* keys, float* range_out,
                          cudaStream_t stream) {
    const int npix = P.rows * P.cols;
    flic_decode_kernel<<<blocks_for(npix, 256), 256, 0, stream>>>(keys, npix, range_out);
    return cudaGetLastError();
}

// Blocks along x of a batched launch: enough for the largest item, at most a few waves of
// the GPU over all items.
static int batch_blocks_x(int max_elems, int nitems, int threads) {
    int bx = (max_elems + threads - 1) / threads;
    const int cap = (152 * 16) / (nitems > 0 ? nitems : 1);
    if (bx > cap) bx = cap;
    return bx < 1 ? 1 : bx;
}

cudaError_t launch_project_batch(const ProjBatch& B, cudaStream_t stream) {
    if (B.nitems <= 0) return cudaSuccess;
    const dim3 gp(batch_blocks_x(B.max_px, B.nitems, 256), B.nitems);
    const dim3 gn(batch_blocks_x(B.max_n, B.nitems, 256), B.nitems);
    flic_clear_keys_batch_kernel<<<gp, 256, 0, stream>>>(B);
    if (B.max_n > 0) flic_project_batch_kernel<<<gn, 256, 0, stream>>>(B);
    flic_decode_batch_kernel<<<gp, 256, 0, stream>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_scatter_batch(const ProjBatch& B, cudaStream_t stream) {
    if (B.nitems <= 0 || B.max_n <= 0) return cudaSuccess;
    const dim3 gn(batch_blocks_x(B.max_n, B.nitems, 256), B.nitems);
    flic_scatter_batch_kernel<<<gn, 256, 0, stream>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const int32_t* labels, int64_t npix, const int32_t* point_pixel,
                           int64_t n, int32_t* point_labels, cudaStream_t stream) {
    if (n > 0) {
        flic_scatter_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(labels, npix, point_pixel, n,
                                                                    point_labels);
    }
    return cudaGetLastError();
}

}  // namespace flic
