// flic_relabel.cu — cluster candidates (§III-B): components with fewer than a minimum
// number of measurements are dropped as sensor noise, the others numbered 0..N-1 by their
// minimum index (the raster order of their first pixels).
//
// The input labels are component minima (flic_label), so a component is identified by its
// root pixel p (labels[p] == p); its size is counted at cnt[p], and later cnt[p] is
// overwritten with its new id.  Six launches over tiles of kRelabelTile pixels of every
// frame (stream-ordered, nothing waits on a flag); the labels are read twice:
//   zero    cnt[p] = 0;
//   hist    cnt[l] += 1 for every pixel labelled l (grouped per warp with __match_any_sync,
//           then per tile in a shared-memory table, one global atomic per label and tile),
//           and the tile's root bitmask (bit p: labels[p] == p), 128 words in raster order;
//   count   per tile, from the root bitmask and the counts at the roots: the kept bitmask
//           (cnt >= min_size) and the number of kept roots;
//   scan    per frame, exclusive offsets of the tiles' counts; N;
//   assign  cnt[p] = the rank of root p among the kept roots of its frame, or -1;
//   apply   labels[p] = cnt[labels[p]].
// A label outside 0..npix-1 (not the output of the labeller) is never used as an index: it
// is left in place and reported in the handle's status word.
#include <cstdint>

#include "flic_internal.h"

namespace flic {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

// The six kernels are launched with programmatic stream serialization: each one waits
// here until the grid before it on the stream has completed and its writes are visible,
// so only the launch of the next grid overlaps the end of the previous one.
__device__ __forceinline__ void wait_prior_grid() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
constexpr int kWords = kRelabelTile / 32;  // bitmask words per tile (128)
static_assert(kRelabelTile == 16 * kThreads, "16 pixels per thread");

__device__ __forceinline__ RelabelFrame frame_at(const RelabelLaunch& L, int f) {
    return L.frames ? L.frames[f] : L.single;
}

__device__ __forceinline__ void report_bad(const RelabelFrame& F) {
    if (F.status) atomicExch(F.status, kRelabelBadLabel);
}

// The frame holding tile t: from the host-built map, or frame 0 of a single-frame launch.
__device__ __forceinline__ int frame_of_tile(const RelabelLaunch& L, int t) {
    return L.tile_frame ? __ldg(L.tile_frame + t) : 0;
}

// Pixels of a tile as thread j sees them in the vector passes: four 16-byte groups,
// p0 + 1024 q + 4 j + e (q, e = 0..3), so that each load of a warp reads 512 contiguous
// bytes.  Frames whose size is not a multiple of 4 (or whose buffers are not 16-byte
// aligned) take the scalar path element by element.
__device__ __forceinline__ bool vec_ok(const RelabelFrame& F) {
    return ((F.npix & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.labels) & 15) == 0) &&
           ((reinterpret_cast<uintptr_t>(F.cnt) & 15) == 0);
}

__device__ __forceinline__ void load4(const RelabelFrame& F, int p, bool vec, int (&v)[4]) {
    if (vec && p + 4 <= F.npix) {
        const int4 x = __ldcg(reinterpret_cast<const int4*>(F.labels + p));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = p + e < F.npix ? __ldcg(F.labels + p + e) : -1;
    }
}

__global__ void __launch_bounds__(kThreads) relabel_zero(const RelabelLaunch L) {
    wait_prior_grid();
    const int t = blockIdx.x;
    const RelabelFrame F = frame_at(L, frame_of_tile(L, t));
    const int p0 = (t - F.tile0) * kRelabelTile;
    const bool vec = vec_ok(F);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int p = p0 + 1024 * q + 4 * threadIdx.x;
        if (vec && p + 4 <= F.npix) {
            __stcg(reinterpret_cast<int4*>(F.cnt + p), make_int4(0, 0, 0, 0));
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (p + e < F.npix) __stcg(F.cnt + p + e, 0);
        }
    }
}

// A tile's counts are gathered in a shared-memory table first (open addressing, a bounded
// probe; a label that finds no slot goes straight to global memory).
constexpr int kHistSlots = 1024;

__global__ void __launch_bounds__(kThreads) relabel_hist(const RelabelLaunch L) {
    wait_prior_grid();
    __shared__ int keys[kHistSlots];
    __shared__ int vals[kHistSlots];
    const int t = blockIdx.x;
    const RelabelFrame F = frame_at(L, frame_of_tile(L, t));
    const int p0 = (t - F.tile0) * kRelabelTile;
    const int lane = threadIdx.x & 31;
    const bool vec = vec_ok(F);
    for (int i = threadIdx.x; i < kHistSlots; i += kThreads) {
        keys[i] = -1;
        vals[i] = 0;
    }
    int v[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) load4(F, p0 + 1024 * q + 4 * threadIdx.x, vec, v[q]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int pq = p0 + 1024 * q + 4 * threadIdx.x;
        unsigned nib = 0;  // root bits of this thread's four pixels
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int l = v[q][e];
            if (l >= F.npix) {
                report_bad(F);
                l = -1;
            }
            if (l == pq + e) nib |= 1u << e;
            const unsigned grp = __match_any_sync(kFull, l);
            if (l >= 0 && lane == __ffs(grp) - 1) {
                const int n = __popc(grp);
                unsigned h = ((unsigned)l * 0x9E3779B1u) >> 22;  // 10 bits
                bool done = false;
                for (int probe = 0; probe < 16; ++probe, h = (h + 1) & (kHistSlots - 1)) {
                    const int k = atomicCAS(keys + h, -1, l);
                    if (k == -1 || k == l) {
                        atomicAdd(vals + h, n);
                        done = true;
                        break;
                    }
                }
                if (!done) atomicAdd(F.cnt + l, n);
            }
        }
        // eight lanes make one word: pixel 4 j + e of the group is bit 4 (j % 8) + e
        unsigned w = nib << (4 * (lane & 7));
        w |= __shfl_xor_sync(kFull, w, 1);
        w |= __shfl_xor_sync(kFull, w, 2);
        w |= __shfl_xor_sync(kFull, w, 4);
        if ((lane & 7) == 0) __stcg(L.roots + (size_t)t * kWords + 32 * q + (threadIdx.x >> 3), w);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistSlots; i += kThreads)
        if (keys[i] >= 0) atomicAdd(F.cnt + keys[i], vals[i]);
}

// Two tiles per block: threads 0..127 take the words of tile 2b, threads 128..255 those
// of tile 2b + 1, one bitmask word each (a block per tile left half of its threads idle).
__device__ __forceinline__ int pair_tile(int& wi) {
    const int half = threadIdx.x / kWords;
    wi = threadIdx.x - half * kWords;
    return 2 * blockIdx.x + half;
}

__global__ void __launch_bounds__(kThreads) relabel_count(const RelabelLaunch L) {
    wait_prior_grid();
    __shared__ int red[kThreads / 32];
    int wi;
    const int t = pair_tile(wi);
    const bool live = t < L.ntiles;
    int c = 0;
    if (live) {
        const RelabelFrame F = frame_at(L, frame_of_tile(L, t));
        const int p0 = (t - F.tile0) * kRelabelTile;
        const unsigned r = __ldcg(L.roots + (size_t)t * kWords + wi);
        unsigned k = 0;
        if (r) {  // the counts of the word's roots, all loads in flight at once
            const int32_t* wc = F.cnt + p0 + 32 * wi;
#pragma unroll
            for (int b = 0; b < 32; ++b)
                if (((r >> b) & 1u) && __ldcg(wc + b) >= L.min_size) k |= 1u << b;
        }
        __stcg(L.kept + (size_t)t * kWords + wi, k);
        c = __popc(k);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    if (wi == 0 && live) {  // the first thread of each half sums its tile's four warps
        constexpr int kWarpsPerTile = kWords / 32;
        int s = 0;
        for (int w = 0; w < kWarpsPerTile; ++w) s += red[warp + w];
        L.tile_cnt[t] = s;
    }
}

// One block per frame: exclusive offsets of its tiles' counts (at most 2^21 / kRelabelTile
// = 512 tiles, two per thread), and the frame's total.
__global__ void __launch_bounds__(kThreads) relabel_scan(const RelabelLaunch L) {
    wait_prior_grid();
    __shared__ int part[kThreads];
    const RelabelFrame F = frame_at(L, blockIdx.x);
    const int nt = (F.npix + kRelabelTile - 1) / kRelabelTile;
    const int i0 = 2 * threadIdx.x;
    const int a = i0 < nt ? L.tile_cnt[F.tile0 + i0] : 0;
    const int b = i0 + 1 < nt ? L.tile_cnt[F.tile0 + i0 + 1] : 0;
    part[threadIdx.x] = a + b;
    __syncthreads();
    // inclusive scan of the pair sums (Hillis-Steele, 256 entries)
    for (int o = 1; o < kThreads; o <<= 1) {
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int before = threadIdx.x ? part[threadIdx.x - 1] : 0;
    if (i0 < nt) L.tile_off[F.tile0 + i0] = before;
    if (i0 + 1 < nt) L.tile_off[F.tile0 + i0 + 1] = before + a;
    if (threadIdx.x == kThreads - 1 && F.num_out) *F.num_out = part[kThreads - 1];
}

// Two tiles per block as in relabel_count, one word per thread: an exclusive prefix of the
// kept counts over the tile's words (raster order), then every root of the word gets its
// rank, or -1.
__global__ void __launch_bounds__(kThreads) relabel_assign(const RelabelLaunch L) {
    wait_prior_grid();
    constexpr int kWarpsPerTile = kWords / 32;
    __shared__ int red[kThreads / 32];
    __shared__ int warp_off[kThreads / 32];
    int wi;
    const int t = pair_tile(wi);
    const bool live = t < L.ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RelabelFrame F{};
    int p0 = 0;
    unsigned r = 0, k = 0;
    if (live) {
        F = frame_at(L, frame_of_tile(L, t));
        p0 = (t - F.tile0) * kRelabelTile;
        r = __ldcg(L.roots + (size_t)t * kWords + wi);
        k = __ldcg(L.kept + (size_t)t * kWords + wi);
    }
    const int c = __popc(k);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    if (wi == 0) {  // the first thread of each half: its tile's warp offsets
        int s = 0;
        for (int w = warp; w < warp + kWarpsPerTile; ++w) {
            warp_off[w] = s;
            s += red[w];
        }
    }
    __syncthreads();
    if (!live) return;
    const int base = L.tile_off[t] + warp_off[warp] + incl - c;
    while (r) {
        const int b = __ffs(r) - 1;
        r &= r - 1u;
        const bool kb = (k >> b) & 1u;
        __stcg(F.cnt + p0 + 32 * wi + b, kb ? base + __popc(k & ((1u << b) - 1u)) : -1);
    }
}

__global__ void __launch_bounds__(kThreads) relabel_apply(const RelabelLaunch L) {
    wait_prior_grid();
    const int t = blockIdx.x;
    const RelabelFrame F = frame_at(L, frame_of_tile(L, t));
    const int p0 = (t - F.tile0) * kRelabelTile;
    const bool vec = vec_ok(F);
    int v[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) load4(F, p0 + 1024 * q + 4 * threadIdx.x, vec, v[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int p = p0 + 1024 * q + 4 * threadIdx.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int l = v[q][e];
            // the new id of a component sits at its root; other values are left alone
            if (l >= 0 && l < F.npix) v[q][e] = __ldcg(F.cnt + l);
        }
        if (vec && p + 4 <= F.npix) {
            __stcg(reinterpret_cast<int4*>(F.labels + p),
                   make_int4(v[q][0], v[q][1], v[q][2], v[q][3]));
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (p + e < F.npix) __stcg(F.labels + p + e, v[q][e]);
        }
    }
}

}  // namespace

namespace {

cudaError_t launch_dependent(void (*kernel)(const RelabelLaunch), int grid,
                             const RelabelLaunch& L, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, L);
}

}  // namespace

cudaError_t launch_relabel(const RelabelLaunch& L, cudaStream_t stream, bool counted) {
    if (L.ntiles <= 0) return cudaSuccess;
    cudaError_t e;
    if (counted) {
        // after the labeller's graph: an ordinary stream-ordered launch (its wait is a no-op)
        relabel_count<<<(L.ntiles + 1) / 2, kThreads, 0, stream>>>(L);
        e = cudaGetLastError();
    } else {
        e = launch_dependent(relabel_zero, L.ntiles, L, stream);
        if (e == cudaSuccess) e = launch_dependent(relabel_hist, L.ntiles, L, stream);
        if (e == cudaSuccess) e = launch_dependent(relabel_count, (L.ntiles + 1) / 2, L, stream);
    }
    if (e == cudaSuccess) e = launch_dependent(relabel_scan, L.nframes, L, stream);
    if (e == cudaSuccess) e = launch_dependent(relabel_assign, (L.ntiles + 1) / 2, L, stream);
    if (e == cudaSuccess) e = launch_dependent(relabel_apply, L.ntiles, L, stream);
    return e;
}

}  // namespace flic
