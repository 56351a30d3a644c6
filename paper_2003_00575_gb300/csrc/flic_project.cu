// flic_project.cu — spherical projection of an xyz cloud into the range image and the
// scatter of pixel labels back onto the points (§I, Fig. 1; §IV-B on one-to-one
// point/pixel matching).
//
// Bin membership is decided only by exact fp32 sign tests against boundary vectors built
// on the host in double and rounded once:
//   column c  iff  cos(c d)*y - sin(c d)*x >= 0  and  cos((c+1) d)*y - sin((c+1) d)*x < 0
//   row band j (sorted boundaries m_j < m_j+1)  iff  cos(m_j)*z - sin(m_j)*rho >= 0 and
//                                                    cos(m_j+1)*z - sin(m_j+1)*rho < 0
// A polynomial azimuth and a table of tan(elevation) buckets only seed the two searches;
// the answer never depends on their rounding.
// Each product, sum and square root is a separately rounded fp32 operation.
// A pixel keeps the smallest range of the points that land in it: one 32-bit atomicMin on
// the range's bits (positive finite floats order like their bits; all bits set = empty).
// Which of several equal ranges wins is not observable, so the key holds no point index.
#include <cstdint>

#include "flic_device.cuh"
#include "flic_internal.h"

namespace flic {

namespace {

constexpr float kTwoPiF = 6.28318530717958647692f;

// Sign of the point against boundary j (row) or column c: cos * z - sin * rho and
// cos * y - sin * x, the (cos, sin) pair read as one 8-byte load.
__device__ __forceinline__ float s_col(const float* __restrict__ colb, int C, int c, float x,
                                       float y) {
    const int i = c >= C ? c - C : c;
    const float2 cs = __ldg(reinterpret_cast<const float2*>(colb) + i);
    return __fsub_rn(__fmul_rn(cs.x, y), __fmul_rn(cs.y, x));
}

__device__ __forceinline__ float s_row(const float* __restrict__ rowb, int j, float z,
                                       float rho) {
    const float2 cs = __ldg(reinterpret_cast<const float2*>(rowb) + j);
    return __fsub_rn(__fmul_rn(cs.x, z), __fmul_rn(cs.y, rho));
}

// Seed of the azimuth search: atan2(y, x) in [0, 2 pi] within about 1.1e-6 rad, from an
// octant reduction and atan(q) ~ q P(q^2) on [0, 1], P of degree 6 with coefficients from
// an iteratively reweighted least-squares fit toward the minimax error (3.3e-7 rad as
// evaluated in fp32).  It decides a column only where the handle's margin makes the sign
// tests' answer known.
__device__ __forceinline__ float azimuth_seed(float x, float y) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float q = __fdividef(fminf(ax, ay), fmaxf(ax, ay));
    const float u = __fmul_rn(q, q);
    float p = __fmaf_rn(u, 0.006812733132392168f, -0.03360702842473984f);
    p = __fmaf_rn(p, u, 0.07962686568498611f);
    p = __fmaf_rn(p, u, -0.1323351413011551f);
    p = __fmaf_rn(p, u, 0.19807860255241394f);
    p = __fmaf_rn(p, u, -0.3331737220287323f);
    p = __fmaf_rn(p, u, 0.9999961256980896f);
    float a = __fmul_rn(p, q);
    if (ay > ax) a = __fsub_rn(1.57079632679489662f, a);
    if (x < 0.0f) a = __fsub_rn(3.14159265358979324f, a);
    if (y < 0.0f) a = __fsub_rn(kTwoPiF, a);
    return a;
}

// Asks L2 for bytes [p, min(p + bytes, end)) of a buffer ahead of their use (16-byte
// granules; p and end 16-byte aligned).  One thread of a block issues it for the slice the
// whole block reads a few iterations later, so that many more bytes are in flight than
// the block's registers could hold.
__device__ __forceinline__ void prefetch_l2(const void* p, const void* end, uint32_t bytes) {
    const uintptr_t a = (uintptr_t)p, e = (uintptr_t)end;
    if (a >= e) return;
    uint32_t n = (uint32_t)((e - a < bytes ? e - a : bytes) & ~(uintptr_t)15);
    if (n == 0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
}

constexpr int kPrefetchAhead = 2;  // iterations of a block's grid-stride loop

// The bins.  A point's row band lo is the one with s(lo) >= 0 and s(lo + 1) < 0, and its
// column c the one with s(c) >= 0 and s(c + 1) < 0 (modulo cols).  Each search starts
// from a seed: the handle's tan(elevation) bucket and azimuth_seed.  Where the seed places
// the point farther than the handle's margins from every boundary that could matter (its
// t outside the bucket's [tlo, thi]; a column fraction inside the column margin) the bin
// is the answer of the sign tests, which then are not evaluated; otherwise the sign tests
// settle it, a point that climbs past the top boundary or falls below the bottom one
// lying outside the field.  A handle without a seed table (an outer boundary beyond +-80
// degrees) bisects between the two outer tests instead.

// Row of a point whose bucket is not certain, settled from the bucket's band lo (-1
// outside the field); settled = false when the walk gave up.
__device__ __forceinline__ int settle_row(const ProjDesc& P, float z, float rho2, int lo,
                                          bool& settled) {
    const float rho = __fsqrt_rn(rho2);
    for (int it = 0; it <= P.rows; ++it) {
        if (s_row(P.rowb, lo + 1, z, rho) >= 0.0f) {
            if (lo + 1 == P.rows) return -1;  // above the top boundary
            ++lo;
        } else if (s_row(P.rowb, lo, z, rho) < 0.0f) {
            if (lo == 0) return -1;           // below the bottom boundary
            --lo;
        } else {
            return __ldg(P.srow + lo);
        }
    }
    settled = false;
    return __ldg(P.srow + lo);
}

__device__ __forceinline__ int settle_col(const ProjDesc& P, float x, float y, int c,
                                          bool& settled) {
    for (int it = 0; it < 64; ++it) {
        if (s_col(P.colb, P.cols, c + 1, x, y) >= 0.0f) {
            c = c + 1 == P.cols ? 0 : c + 1;
        } else if (s_col(P.colb, P.cols, c, x, y) < 0.0f) {
            c = c == 0 ? P.cols - 1 : c - 1;
        } else {
            return c;
        }
    }
    settled = false;
    return c;
}

// Pixels of N points of a cloud on a handle with a seed table: the arithmetic of all N
// first, then their N table loads at once, then the rare settles, the pixels and the keys
// offered to them (the smallest range wins).  Every index computed from a point that is no
// measurement stays in bounds (NaN converts to 0; the bucket and column are clamped) and
// is not used.
template <int N>
__device__ __forceinline__ void project_group(const ProjDesc& P, const RowSeed* seeds,
                                              const float (&x)[N], const float (&y)[N],
                                              const float (&z)[N],
                                              uint32_t* __restrict__ keys,
                                              int32_t (&out)[N]) {
    float rg[N], rho2[N], fr[N], t[N];
    int b[N], c[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        rho2[j] = __fadd_rn(__fmul_rn(x[j], x[j]), __fmul_rn(y[j], y[j]));
        rg[j] = __fsqrt_rn(__fadd_rn(rho2[j], __fmul_rn(z[j], z[j])));
        t[j] = __fmul_rn(z[j], rsqrtf(rho2[j]));
        const float fb = (t[j] - P.rs_t0) * P.rs_inv_dt;
        b[j] = (int)fminf(fmaxf(fb, 0.0f), (float)(kRowSeeds - 1));
        const float fc = __fmul_rn(azimuth_seed(x[j], y[j]), P.inv_az_step);
        int cc = (int)fc;
        cc = cc < 0 ? 0 : (cc >= P.cols ? P.cols - 1 : cc);
        c[j] = cc;
        fr[j] = __fsub_rn(fc, (float)cc);
    }
    RowSeed e[N];
#pragma unroll
    for (int j = 0; j < N; ++j) e[j] = seeds[b[j]];
    const float hi = __fsub_rn(1.0f, P.col_margin);
    bool settled = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        int32_t pix = -1;
        if (valid_range(rg[j]) && rho2[j] > 0.0f) {
            int row;
            if (t[j] < e[j].tlo) {
                row = (int)((e[j].info >> 10) & 1023u);
            } else if (t[j] > e[j].thi) {
                row = (int)((e[j].info >> 20) & 1023u);
            } else {
                row = settle_row(P, z[j], rho2[j], (int)(e[j].info & 1023u), settled);
                if (row < 0) row = (int)kRowOutside;
            }
            if (row != (int)kRowOutside) {
                int cc = c[j];
                if (!(fr[j] > P.col_margin && fr[j] < hi)) cc = settle_col(P, x[j], y[j], cc, settled);
                pix = row * P.cols + cc;
                atomicMin(keys + pix, __float_as_uint(rg[j]));
            }
        }
        out[j] = pix;
    }
    if (!settled) report_timeout(P.status);
}

// The same bins on a handle without a seed table: bisection between the outer boundaries.
__device__ __forceinline__ int32_t pixel_of_bisect(const ProjDesc& P, float x, float y, float z,
                                                   uint32_t* __restrict__ keys) {
    const float rho2 = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
    const float rg = __fsqrt_rn(__fadd_rn(rho2, __fmul_rn(z, z)));
    if (!valid_range(rg) || !(rho2 > 0.0f)) return -1;
    const float rho = __fsqrt_rn(rho2);
    if (!(s_row(P.rowb, 0, z, rho) >= 0.0f) || !(s_row(P.rowb, P.rows, z, rho) < 0.0f))
        return -1;
    int lo = 0, hi = P.rows;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_row(P.rowb, mid, z, rho) >= 0.0f) lo = mid; else hi = mid;
    }
    int c = (int)(azimuth_seed(x, y) * P.inv_az_step);
    c = c < 0 ? 0 : (c >= P.cols ? P.cols - 1 : c);
    bool settled = true;
    c = settle_col(P, x, y, c, settled);
    if (!settled) report_timeout(P.status);
    const int32_t pix = __ldg(P.srow + lo) * P.cols + c;
    atomicMin(keys + pix, __float_as_uint(rg));
    return pix;
}

__device__ __forceinline__ int32_t project_one(const ProjDesc& P, const RowSeed* seeds,
                                               const float* __restrict__ xyz, int64_t i,
                                               uint32_t* __restrict__ keys) {
    const float x = __ldg(xyz + 3 * i), y = __ldg(xyz + 3 * i + 1), z = __ldg(xyz + 3 * i + 2);
    if (!(P.rs_inv_dt > 0.0f)) return pixel_of_bisect(P, x, y, z, keys);
    const float xs[1] = {x}, ys[1] = {y}, zs[1] = {z};
    int32_t out[1];
    project_group<1>(P, seeds, xs, ys, zs, keys, out);
    return out[0];
}

// Points [first, n) of a cloud in steps of stride, four per thread from three 16-byte loads
// (the next four already in flight) where xyz and point_pixel are 16-byte aligned.
__device__ __forceinline__ void project_points(const ProjDesc& P, const RowSeed* seeds,
                                               const float* __restrict__ xyz,
                                               int64_t n, uint32_t* __restrict__ keys,
                                               int32_t* __restrict__ point_pixel, int64_t first,
                                               int64_t stride) {
    int64_t done = 0;
    if ((((uintptr_t)xyz | (uintptr_t)point_pixel) & 15) == 0 && P.rs_inv_dt > 0.0f) {
        const int64_t n4 = n >> 2;
        const float4* __restrict__ x4 = reinterpret_cast<const float4*>(xyz);
        int64_t g = first;
        const bool lead = threadIdx.x == 0;  // the block's lowest group: iterates longest
        const float4* end4 = x4 + 3 * n4;
        if (lead)
            for (int d = 1; d <= kPrefetchAhead; ++d)
                prefetch_l2(x4 + 3 * (g + d * stride), end4, 48u * blockDim.x);
        float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), b = a, c = a;
        if (g < n4) {
            a = __ldg(x4 + 3 * g);
            b = __ldg(x4 + 3 * g + 1);
            c = __ldg(x4 + 3 * g + 2);
        }
        while (g < n4) {
            const int64_t gn = g + stride;
            if (lead) prefetch_l2(x4 + 3 * (g + (kPrefetchAhead + 1) * stride), end4,
                                  48u * blockDim.x);
            float4 na = a, nb = b, nc = c;
            if (gn < n4) {
                na = __ldg(x4 + 3 * gn);
                nb = __ldg(x4 + 3 * gn + 1);
                nc = __ldg(x4 + 3 * gn + 2);
            }
            const float xs[4] = {a.x, a.w, b.z, c.y};
            const float ys[4] = {a.y, b.x, b.w, c.z};
            const float zs[4] = {a.z, b.y, c.x, c.w};
            int32_t o[4];
            project_group<4>(P, seeds, xs, ys, zs, keys, o);
            reinterpret_cast<int4*>(point_pixel)[g] = make_int4(o[0], o[1], o[2], o[3]);
            a = na;
            b = nb;
            c = nc;
            g = gn;
        }
        done = 4 * n4;
    }
    for (int64_t i = done + first; i < n; i += stride)
        point_pixel[i] = project_one(P, seeds, xyz, i, keys);
}

// keys[0, npix) <- empty, four keys per 16-byte store where aligned
__device__ __forceinline__ void clear_keys(uint32_t* __restrict__ keys, int64_t npix,
                                           int64_t first, int64_t stride) {
    int64_t done = 0;
    if (((uintptr_t)keys & 15) == 0) {
        const int64_t n4 = npix >> 2;
        for (int64_t p = first; p < n4; p += stride)
            reinterpret_cast<uint4*>(keys)[p] = make_uint4(~0u, ~0u, ~0u, ~0u);
        done = 4 * n4;
    }
    for (int64_t p = done + first; p < npix; p += stride) keys[p] = ~0u;
}

// range_out[p] <- the smallest range of pixel p (0 where no point landed), four pixels per
// 16-byte access where aligned.
__device__ __forceinline__ float key_range(uint32_t k) {
    return k == ~0u ? 0.0f : __uint_as_float(k);
}

__device__ __forceinline__ void decode_keys(const uint32_t* __restrict__ keys, int64_t npix,
                                            float* __restrict__ range_out, int64_t first,
                                            int64_t stride) {
    int64_t done = 0;
    if ((((uintptr_t)keys | (uintptr_t)range_out) & 15) == 0) {
        const int64_t n4 = npix >> 2;
        const uint4* k4 = reinterpret_cast<const uint4*>(keys);
        const bool lead = threadIdx.x == 0;
        if (lead)
            for (int d = 1; d <= kPrefetchAhead; ++d)
                prefetch_l2(k4 + first + d * stride, k4 + n4, 16u * blockDim.x);
        for (int64_t p = first; p < n4; p += stride) {
            if (lead) prefetch_l2(k4 + p + (kPrefetchAhead + 1) * stride, k4 + n4, 16u * blockDim.x);
            const uint4 a = __ldcs(k4 + p);
            reinterpret_cast<float4*>(range_out)[p] =
                make_float4(key_range(a.x), key_range(a.y), key_range(a.z), key_range(a.w));
        }
        done = 4 * n4;
    }
    for (int64_t p = done + first; p < npix; p += stride) range_out[p] = key_range(keys[p]);
}

// point_labels[i] <- labels[point_pixel[i]] (-1 for a point without a pixel), four points
// per thread from 16-byte loads and stores where aligned (four gathers in flight).
__device__ __forceinline__ int32_t label_at(const int32_t* __restrict__ labels, int64_t npix,
                                            int32_t p) {
    return (p >= 0 && p < npix) ? __ldg(labels + p) : -1;
}

__device__ __forceinline__ void scatter_points(const int32_t* __restrict__ labels, int64_t npix,
                                               const int32_t* __restrict__ point_pixel, int64_t n,
                                               int32_t* __restrict__ point_labels, int64_t first,
                                               int64_t stride) {
    int64_t done = 0;
    if ((((uintptr_t)point_pixel | (uintptr_t)point_labels) & 15) == 0) {
        const int64_t n4 = n >> 2;
        const int4* p4 = reinterpret_cast<const int4*>(point_pixel);
        const bool lead = threadIdx.x == 0;
        if (lead)
            for (int d = 1; d <= kPrefetchAhead; ++d)
                prefetch_l2(p4 + first + d * stride, p4 + n4, 16u * blockDim.x);
        for (int64_t g = first; g < n4; g += stride) {
            if (lead) prefetch_l2(p4 + g + (kPrefetchAhead + 1) * stride, p4 + n4, 16u * blockDim.x);
            const int4 p = __ldcs(p4 + g);
            int4 o;
            o.x = label_at(labels, npix, p.x);
            o.y = label_at(labels, npix, p.y);
            o.z = label_at(labels, npix, p.z);
            o.w = label_at(labels, npix, p.w);
            reinterpret_cast<int4*>(point_labels)[g] = o;
        }
        done = 4 * n4;
    }
    for (int64_t i = done + first; i < n; i += stride)
        point_labels[i] = label_at(labels, npix, __ldg(point_pixel + i));
}

// The handle's seed table, staged once per block in shared memory (kSeedBytes of dynamic
// shared memory) or read through L1 in place.
constexpr bool kSeedsInShared = true;
constexpr size_t kSeedBytes = kSeedsInShared ? sizeof(RowSeed) * kRowSeeds : 0;
static_assert(sizeof(RowSeed) == 16, "one seed per 16-byte copy");

__device__ __forceinline__ const RowSeed* stage_seeds(const ProjDesc& P) {
    if (!kSeedsInShared || !(P.rs_inv_dt > 0.0f)) return P.rseed;
    extern __shared__ uint4 seed_smem[];
    const uint4* src = reinterpret_cast<const uint4*>(P.rseed);
    for (int i = threadIdx.x; i < kRowSeeds; i += blockDim.x) seed_smem[i] = __ldg(src + i);
    __syncthreads();
    return reinterpret_cast<const RowSeed*>(seed_smem);
}

__global__ void flic_project_kernel(const ProjDesc P, const float* __restrict__ xyz, int64_t n,
                                    uint32_t* __restrict__ keys,
                                    int32_t* __restrict__ point_pixel) {
    const RowSeed* seeds = stage_seeds(P);
    project_points(P, seeds, xyz, n, keys, point_pixel,
                   (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

__global__ void flic_decode_kernel(const uint32_t* __restrict__ keys, int npix,
                                   float* __restrict__ range_out) {
    decode_keys(keys, npix, range_out, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
}

// ---- many clouds per launch: blockIdx.y is the item, x strides over its points or pixels

__global__ void flic_clear_keys_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    clear_keys(it.keys, (int64_t)it.P.rows * it.P.cols, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

__global__ void flic_project_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    const RowSeed* seeds = stage_seeds(it.P);
    project_points(it.P, seeds, it.xyz, it.n, it.keys, it.point_pixel,
                   blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void flic_decode_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    decode_keys(it.keys, (int64_t)it.P.rows * it.P.cols, it.range_out,
                blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void flic_scatter_batch_kernel(const ProjBatch B) {
    const ProjItem& it = B.item[blockIdx.y];
    scatter_points(it.labels, (int64_t)it.P.rows * it.P.cols, it.point_pixel, it.n,
                   it.point_labels, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void flic_scatter_kernel(const int32_t* __restrict__ labels, int64_t npix,
                                    const int32_t* __restrict__ point_pixel, int64_t n,
                                    int32_t* __restrict__ point_labels) {
    scatter_points(labels, npix, point_pixel, n, point_labels,
                   (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

cudaError_t launch_project(const ProjDesc& P, const float* xyz, int64_t n, uint32_t* keys,
                           int32_t* point_pixel, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(keys, 0xff, sizeof(uint32_t) * (size_t)P.rows *
                                                    (size_t)P.cols, stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        flic_project_kernel<<<blocks_for((n + 3) / 4, 256), 256, kSeedBytes, stream>>>(
            P, xyz, n, keys, point_pixel);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode(const ProjDesc& P, const uint32_t* keys, float* range_out,
                          cudaStream_t stream) {
    const int npix = P.rows * P.cols;
    flic_decode_kernel<<<blocks_for((npix + 3) / 4, 256), 256, 0, stream>>>(keys, npix, range_out);
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
    const dim3 gp(batch_blocks_x((B.max_px + 3) / 4, B.nitems, 256), B.nitems);  // 4 px/thread
    const dim3 gn(batch_blocks_x((B.max_n + 3) / 4, B.nitems, 256), B.nitems);   // 4 points
    flic_clear_keys_batch_kernel<<<gp, 256, 0, stream>>>(B);
    if (B.max_n > 0) flic_project_batch_kernel<<<gn, 256, kSeedBytes, stream>>>(B);
    flic_decode_batch_kernel<<<gp, 256, 0, stream>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_scatter_batch(const ProjBatch& B, cudaStream_t stream) {
    if (B.nitems <= 0 || B.max_n <= 0) return cudaSuccess;
    const dim3 gn(batch_blocks_x((B.max_n + 3) / 4, B.nitems, 256), B.nitems);  // 4 points
    flic_scatter_batch_kernel<<<gn, 256, 0, stream>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const int32_t* labels, int64_t npix, const int32_t* point_pixel,
                           int64_t n, int32_t* point_labels, cudaStream_t stream) {
    if (n > 0) {
        flic_scatter_kernel<<<blocks_for((n + 3) / 4, 256), 256, 0, stream>>>(
            labels, npix, point_pixel, n, point_labels);
    }
    return cudaGetLastError();
}

}  // namespace flic
