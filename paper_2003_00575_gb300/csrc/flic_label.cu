// flic_label.cu — the FLIC neighbour test and connected-component labelling on sm_103a.
//
// One thread-block cluster labels one work item: up to kMaxCluster full-height column
// strips of one or more frames.  Each block owns one strip (rows x W columns) and runs:
//
//   phase 1  (edge test + tile-local union, in shared memory)
//            a. each warp takes a 32-column row segment; the horizontal offset-1 edge
//               bits (Eq. 2/3) of the segment are gathered with __ballot_sync and every
//               pixel's parent is set to the first pixel of its run, so a run of joined
//               pixels becomes one star without a single atomic;
//            b. the remaining edges — offset-1 links across segment borders, offsets
//               2..S along the row (Map Connections, §III-B-2) and offsets 1..S down the
//               column — are tested; an edge whose two ends are already joined by runs
//               is dropped with ballot bit tricks, lanes asking for the same union are
//               merged with __match_any_sync, and the rest hook with shared-memory
//               atomicMin (the smaller index becomes the root);
//            c. paths are compressed, so every pixel points at its strip-local root,
//               the minimum index of its strip-local component;
//            d. pixels in the first S columns publish their root in the frame's labels
//               buffer, and roots of components touching either strip border publish
//               themselves: these entries form the cross-strip forest.
//   cluster barrier
//   phase 2  (boundary merge, global memory): every edge that leaves the strip on the
//            right (offsets 1..S, including the azimuth wrap from the last column to the
//            first) unites the two roots with atomicMin hooking and path halving.
//   cluster barrier
//   phase 3  (flatten): roots of border components look up their global root (read-only);
//            every pixel then writes label = the minimum linear index of its component,
//            or -1 for pixels that are not measurements.
//
// The labels buffer is the only global working memory: no scratch allocation.  No block
// ever waits on another except at the two hardware cluster barriers, so the kernel has no
// spin loop; every union and find loop is bounded by an iteration budget whose exhaustion
// sets the frame's status word.
#include <cstdint>

#include "flic_device.cuh"
#include "flic_internal.h"

namespace flic {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Strip {
    const float* range;   // frame origin
    int32_t* labels;
    const float* kv;
    const float* kh;
    int32_t* status;
    int R, C, S;
    float delta2;
    bool wrap;
    bool border;   // edges can leave the strip (several strips or wrap-around)
    int c0, W;     // first column and width of the strip
    int sh;        // local pitch = 1 << sh (>= 32, >= W)
    int limit;
};

__device__ __forceinline__ int global_of(const Strip& s, int local) {
    return (local >> s.sh) * s.C + s.c0 + (local & ((1 << s.sh) - 1));
}

// Union two pixels of the strip unless another lane of the warp asks for the same union
// (same current parents of both ends).  All 32 lanes of the warp must call it.
__device__ __forceinline__ void warp_union(int* par, bool need, int i, int j, int lane,
                                           const Strip& s) {
    unsigned nm = __ballot_sync(kFull, need);
    if (nm == 0) return;
    if (__popc(nm) > 1) {
        // parents < 2^15, so a real key never equals the idle-lane key
        unsigned key = need ? ((unsigned(par[i]) << 16) | unsigned(par[j])) : kFull;
        unsigned grp = __match_any_sync(kFull, key);
        if (need && (__ffs(grp) - 1) != lane) need = false;
    }
    if (need) {
        int budget = s.limit;
        union_smem(par, i, j, budget);
        if (budget <= 0) report_timeout(s.status);
    }
}

__device__ void phase1_local(const Strip& s, int* par, unsigned* hmask) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int P = 1 << s.sh;
    const int segs_log2 = s.sh - 5;
    const int nunits = s.R << segs_log2;

    // a. runs of horizontally joined pixels become stars
    for (int u = warp; u < nunits; u += nwarps) {
        const int r = u >> segs_log2;
        const int seg = u & ((1 << segs_log2) - 1);
        const int c = (seg << 5) + lane;
        const float* rp = s.range + (size_t)r * s.C + s.c0;
        const float a = c < s.W ? load_range(rp + c) : 0.0f;
        const float b = c + 1 < s.W ? load_range(rp + c + 1) : 0.0f;
        const bool h1 = a > 0.0f && b > 0.0f && edge_pred(a, b, __ldg(s.kh + r * s.S), s.delta2);
        const unsigned m = __ballot_sync(kFull, h1);
        if (lane == 0) hmask[u] = m;
        // first lane of this lane's run: one past the highest missing link below it
        const unsigned below = ~m & ((1u << lane) - 1u);
        const int start = below ? 32 - __clz(below) : 0;
        par[(r << s.sh) + c] = a > 0.0f ? (r << s.sh) + (seg << 5) + start : -1;
    }
    __syncthreads();

    // b. every other edge inside the strip
    for (int u = warp; u < nunits; u += nwarps) {
        const int r = u >> segs_log2;
        const int seg = u & ((1 << segs_log2) - 1);
        const int c = (seg << 5) + lane;
        const float* rp = s.range + (size_t)r * s.C + s.c0;
        const float a = c < s.W ? load_range(rp + c) : 0.0f;
        const bool va = a > 0.0f;
        const unsigned m = hmask[u];
        const int i = (r << s.sh) + c;

        // offset-1 link from the last lane into the next segment (h1 implies c + 1 < W)
        {
            const bool need = lane == 31 && ((m >> 31) & 1u);
            warp_union(par, need, i, i + 1, lane, s);
        }
        // offsets 2..S along the row
        for (int k = 2; k <= s.S; ++k) {
            bool e = false;
            if (va && c + k < s.W) {
                const float b = load_range(rp + c + k);
                e = b > 0.0f && edge_pred(a, b, __ldg(s.kh + r * s.S + k - 1), s.delta2);
            }
            if (e && lane + k <= 31) {
                const unsigned run = (m >> lane) & ((1u << k) - 1u);
                if (run == (1u << k) - 1u) e = false;  // same run already
            }
            warp_union(par, e, i, i + k, lane, s);
        }
        // offsets 1..S down the column
        for (int k = 1; k <= s.S && r + k < s.R; ++k) {
            bool e = false;
            if (va) {
                const float b = load_range(rp + (size_t)k * s.C + c);
                e = b > 0.0f && edge_pred(a, b, __ldg(s.kv + r * s.S + k - 1), s.delta2);
            }
            const unsigned em = __ballot_sync(kFull, e);
            const unsigned mk = hmask[u + (k << segs_log2)];
            // lane l is implied by lane l-1 when l-1 has the same vertical edge and both
            // rows join l-1 to l by a horizontal offset-1 edge
            const unsigned implied = (em & m & mk) << 1;
            const bool need = e && !((implied >> lane) & 1u);
            warp_union(par, need, i, i + (k << s.sh), lane, s);
        }
    }
    __syncthreads();

    // c. compress: every measurement points at its strip-local root (read-only finds;
    //    each thread stores only its own entries)
    {
        volatile int* vp = par;
        for (int i = threadIdx.x; i < (s.R << s.sh); i += blockDim.x) {
            if (vp[i] >= 0) {
                int budget = s.limit;
                const int root = find_smem_ro(vp, i, budget);
                if (budget <= 0) report_timeout(s.status);
                vp[i] = root;
            }
        }
    }
    __syncthreads();

    // d. publish the border pixels and border roots into the cross-strip forest
    if (s.border) {
        const int nb = s.S < s.W ? s.S : s.W;   // border columns on each side
        const int per_row = 2 * nb;
        for (int t = threadIdx.x; t < s.R * per_row; t += blockDim.x) {
            const int r = t / per_row;
            const int j = t - r * per_row;
            const int c = j < nb ? j : s.W - per_row + j;  // first nb, then last nb columns
            const int p = par[(r << s.sh) + c];
            if (p < 0) continue;
            const int groot = global_of(s, p);
            if (j < nb) __stcg(s.labels + (size_t)r * s.C + s.c0 + c, groot);
            __stcg(s.labels + groot, groot);
        }
    }
    (void)P;
}

__device__ void phase2_merge(const Strip& s, const int* par) {
    if (!s.border) return;
    const int first = s.W - s.S > 0 ? s.W - s.S : 0;
    const int ncols = s.W - first;
    const int n = s.R * ncols * s.S;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int k = t % s.S + 1;
        const int rc = t / s.S;
        const int r = rc / ncols;
        const int c = first + (rc - r * ncols);
        if (c + k < s.W) continue;  // stays inside the strip: phase 1 handled it
        int tc = s.c0 + c + k;
        if (tc >= s.C) {
            if (!s.wrap) continue;
            tc %= s.C;
        }
        const float a = load_range(s.range + (size_t)r * s.C + s.c0 + c);
        if (!(a > 0.0f)) continue;
        const float b = load_range(s.range + (size_t)r * s.C + tc);
        if (!(b > 0.0f)) continue;
        if (!edge_pred(a, b, __ldg(s.kh + r * s.S + k - 1), s.delta2)) continue;
        const int ga = global_of(s, par[(r << s.sh) + c]);
        const int gb = __ldcg(s.labels + (size_t)r * s.C + tc);
        int budget = s.limit;
        union_global(s.labels, ga, gb, budget);
        if (budget <= 0) report_timeout(s.status);
    }
}

__device__ void phase3_flatten(const Strip& s, int* par) {
    if (s.border) {
        // roots of border components: global root, stored as the tag -(root + 2)
        const int nb = s.S < s.W ? s.S : s.W;
        const int per_row = 2 * nb;
        for (int t = threadIdx.x; t < s.R * per_row; t += blockDim.x) {
            const int r = t / per_row;
            const int j = t - r * per_row;
            const int c = j < nb ? j : s.W - per_row + j;
            const int p = par[(r << s.sh) + c];
            if (p < 0) continue;  // not a measurement, or a root already tagged
            const int groot = global_of(s, p);
            int budget = s.limit;
            const int fin = find_global(s.labels, groot, budget, false);
            if (budget <= 0) report_timeout(s.status);
            if (fin != groot) par[p] = -(fin + 2);
        }
        __syncthreads();
    }
    // every pixel of the strip: 4 consecutive columns per thread
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const bool vec = ((s.C & 3) == 0) && ((s.c0 & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(s.labels) & 15) == 0);
    for (int r = warp; r < s.R; r += nwarps) {
        int32_t* out = s.labels + (size_t)r * s.C + s.c0;
        const int base = r << s.sh;
        for (int c = lane * 4; c < s.W; c += 128) {
            int v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int x = -1;
                if (c + q < s.W) {
                    const int p = par[base + c + q];
                    if (p <= -2) {
                        x = -(p + 2);
                    } else if (p >= 0) {
                        const int w = par[p];
                        x = w <= -2 ? -(w + 2) : global_of(s, p);
                    }
                }
                v[q] = x;
            }
            if (vec && c + 4 <= s.W) {
                __stcs(reinterpret_cast<int4*>(out + c), make_int4(v[0], v[1], v[2], v[3]));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c + q < s.W) out[c + q] = v[q];
            }
        }
    }
}

__global__ void __launch_bounds__(1024) flic_label_kernel(const LabelLaunch L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* par = reinterpret_cast<int*>(smem_raw);

    const unsigned rank = cluster_ctarank();
    const int nitems = L.items ? L.nitems : 1;
    // every block of a cluster walks the same item sequence, so the cluster barriers
    // below are reached the same number of times by all of them
    for (int item = (int)cluster_index(); item < nitems; item += (int)cluster_count()) {
        int fi, si;
        if (L.items) {
            fi = L.items[item].frame[rank];
            si = L.items[item].strip[rank];
        } else {
            fi = (int)rank < L.single.nstrips ? 0 : -1;
            si = (int)rank;
        }
        Strip s{};
        const bool active = fi >= 0;
        if (active) {
            const FrameDesc& f = L.frames ? L.frames[fi] : L.single;
            s.range = f.range;
            s.labels = f.labels;
            s.kv = f.kv;
            s.kh = f.kh;
            s.status = f.status;
            s.R = f.rows;
            s.C = f.cols;
            s.S = f.skip;
            s.delta2 = f.delta2;
            s.wrap = f.wrap != 0;
            s.border = f.nstrips > 1 || s.wrap;
            s.c0 = si * f.strip_w;
            s.W = min(f.strip_w, s.C - s.c0);
            s.sh = f.pitch_log2;
            s.limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
        }
        unsigned* hmask = reinterpret_cast<unsigned*>(par + (active ? (s.R << s.sh) : 0));

        if (active) phase1_local(s, par, hmask);
        __threadfence();
        cluster_barrier();
        if (active) phase2_merge(s, par);
        __threadfence();
        cluster_barrier();
        if (active) phase3_flatten(s, par);
        __syncthreads();  // shared memory is reused by the next item
    }
}

// flic_edges: the neighbour test alone, one pixel per thread, straight from global memory.
__global__ void flic_edges_kernel(const FrameDesc f, uint16_t* __restrict__ mask) {
    const int N = f.rows * f.cols;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int r = p / f.cols;
        const int c = p - r * f.cols;
        const float a = load_range(f.range + p);
        unsigned m = 0;
        if (a > 0.0f) {
            for (int k = 1; k <= f.skip; ++k) {
                int cc = c + k;
                bool has = true;
                if (cc >= f.cols) {
                    if (f.wrap) cc %= f.cols; else has = false;
                }
                if (has) {
                    const float b = load_range(f.range + (size_t)r * f.cols + cc);
                    if (b > 0.0f && edge_pred(a, b, __ldg(f.kh + r * f.skip + k - 1), f.delta2))
                        m |= 1u << (k - 1);
                }
                if (r + k < f.rows) {
                    const float b = load_range(f.range + p + (size_t)k * f.cols);
                    if (b > 0.0f && edge_pred(a, b, __ldg(f.kv + r * f.skip + k - 1), f.delta2))
                        m |= 1u << (8 + k - 1);
                }
            }
        }
        mask[p] = (uint16_t)m;
    }
}

}  // namespace

cudaError_t label_kernel_setup(size_t max_smem) {
    cudaError_t e = cudaFuncSetAttribute(flic_label_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)max_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(flic_label_kernel,
                                cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t launch_label(const LabelLaunch& L, int grid_clusters, int threads, size_t smem,
                         cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid_clusters * L.cluster), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, flic_label_kernel, L);
}

cudaError_t max_active_clusters(int cluster, int threads, size_t smem, int* out) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, flic_label_kernel, &cfg);
}

cudaError_t launch_edges(const FrameDesc& f, uint16_t* mask, cudaStream_t stream) {
    const int N = f.rows * f.cols;
    const int threads = 256;
    int blocks = (N + threads - 1) / threads;
    if (blocks < 1) blocks = 1;
    flic_edges_kernel<<<blocks, threads, 0, stream>>>(f, mask);
    return cudaGetLastError();
}

}  // namespace flic
