// flic_label.cu — the FLIC neighbour test and connected-component labelling on sm_103a.
//
// One thread-block cluster labels one work item: up to kMaxCluster full-height column
// strips of one or more frames.  Each block owns one strip (rows x W columns) and runs:
//
//   phase 1  (edge test + tile-local union, in shared memory)
//            0. the strip's range readings, plus S halo columns on the right (wrapping to
//               column 0 at the seam), are staged into shared memory: one TMA bulk copy
//               (cp.async.bulk) per row completing on an mbarrier, or plain loads when the
//               frame is not 16-byte aligned;
//            1. every pixel's 2S edge bits (Eq. 2/3; offsets 1..S right and down, the
//               Map Connections of §III-B-2) are computed from shared memory into a 16-bit
//               mask per pixel; the staged readings are dead afterwards and their space
//               becomes the parent array;
//            a. each warp takes a 32-column row segment; the offset-1 right bits of the
//               segment are gathered with __ballot_sync and every pixel's parent is set to
//               the first pixel of its run, so a run of joined pixels becomes one star
//               without a single atomic;
//            b. the remaining in-strip edges — offset-1 links across segment borders,
//               offsets 2..S along the row and 1..S down the column — are read from the
//               masks; an edge whose two ends are already joined by runs is dropped with
//               ballot bit tricks, lanes asking for the same union are merged with
//               __match_any_sync, and the rest hook with shared-memory atomicMin (the
//               smaller index becomes the root);
//            c. paths are compressed by pointer jumping, so every pixel points at its
//               strip-local root, the minimum index of its strip-local component;
//            d. pixels in the first S columns publish their root in the frame's labels
//               buffer, and roots of components touching either strip border publish
//               themselves: these entries form the cross-strip forest.
//   cluster barrier
//   phase 2  (boundary merge, global memory): every edge that leaves the strip on the
//            right (mask bits of offsets 1..S, including the azimuth wrap from the last
//            column to the first) unites the two roots with atomicMin hooking and path
//            halving.
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
    int RP;        // row pitch of the staged readings (>= W + S, multiple of 4)
    bool bulk;     // rows are 16-byte aligned: stage with TMA bulk copies
    int limit;
};

// Shared-memory carve-up of one strip (byte offsets; see strip_smem_bytes on the host).
struct Carve {
    float* stage;       // R x RP staged readings; reused as the parent array (R x P)
    int* par;
    uint16_t* mask;     // R x P edge bits
    unsigned* hmask;    // R x P/32 ballot words of the offset-1 right bits
    unsigned* vmask;    // R x P/32 ballot words: the pixel is a measurement
};

__device__ __forceinline__ Carve carve(unsigned char* base, const Strip& s) {
    Carve c;
    const int P = 1 << s.sh;
    const int a_words = s.R * (s.RP > P ? s.RP : P);
    c.stage = reinterpret_cast<float*>(base);
    c.par = reinterpret_cast<int*>(base);
    c.mask = reinterpret_cast<uint16_t*>(base + 4 * (size_t)a_words);
    c.hmask = reinterpret_cast<unsigned*>(base + 4 * (size_t)a_words + 2 * (size_t)s.R * P);
    c.vmask = c.hmask + (s.R << (s.sh - 5));
    return c;
}

__device__ __forceinline__ int global_of(const Strip& s, int local) {
    return (local >> s.sh) * s.C + s.c0 + (local & ((1 << s.sh) - 1));
}

// Union of two pixels of the strip (the caller has already dropped redundant requests).
__device__ __forceinline__ void unite(int* par, int a, int b, const Strip& s) {
    int budget = s.limit;
    union_smem(par, a, b, budget);
    if (budget <= 0) report_timeout(s.status);
}

// b. every edge inside the strip that the runs do not already cover.  Each warp walks a
//    band of consecutive rows of one 32-column segment from the top down and keeps, in
//    registers, the labels and edge masks of the S rows above each of its columns.  A
//    run whose vertical edges all reach pixels of one label X (the common case: ground,
//    walls) just hooks its first pixel under X with one atomicMin; only where several
//    labels meet are real unions needed, one per distinct (run, label) pair, found with
//    __match_any_sync.  Edges that leave the band or the segment use plain unions, with
//    the requests a neighbouring lane already covers dropped by ballot bit tricks.
template <int S>
__device__ void phase1_bands(const Strip& s, const Carve& sm) {
    constexpr int kInf = 0x7fffffff;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int segs_log2 = s.sh - 5;
    const int nseg = 1 << segs_log2;
    int* par = sm.par;
    const int band = (s.R * nseg + nwarps - 1) / nwarps;  // rows per band
    const int nbands = (s.R + band - 1) / band;
    const unsigned lane_lt = (1u << lane) - 1u;

    for (int blk = warp; blk < nbands * nseg; blk += nwarps) {
        const int seg = blk & (nseg - 1);
        const int r0 = (blk >> segs_log2) * band;
        const int r1 = min(s.R, r0 + band);
        const int c = (seg << 5) + lane;
        const bool inw = c < s.W;
        int lab[S];        // lab[k-1]: a label (set member) of pixel (r-k, c), -1 if none
        unsigned mab[S];   // mab[k-1]: edge mask of pixel (r-k, c)
#pragma unroll
        for (int k = 0; k < S; ++k) {
            lab[k] = -1;
            mab[k] = 0u;
        }
        for (int r = r0; r < r1; ++r) {
            const int u = (r << segs_log2) + seg;
            const int base = (r << s.sh) + (seg << 5);
            const int i = base + lane;
            const unsigned mk = inw ? sm.mask[i] : 0u;
            const unsigned m = sm.hmask[u];
            const bool va = inw && ((sm.vmask[u] >> lane) & 1u);
            // this lane's run: first lane st, last lane en, lanes runbits
            const unsigned below = ~m & lane_lt;
            const int st = below ? 32 - __clz(below) : 0;
            const unsigned brk = (~m | 0x80000000u) & ~lane_lt;
            const int en = __ffs(brk) - 1;
            const unsigned runbits = (en == 31 ? kFull : ((2u << en) - 1u)) & ~((1u << st) - 1u);
            const int sidx = base + st;

            // labels of the pixels above that a vertical edge joins to this pixel: the
            // smallest in cand, and whether they differ
            int cand = kInf;
            bool multi = false;
#pragma unroll
            for (int k = 1; k <= S; ++k) {
                if (r - k < 0) break;
                if (r - k >= r0) {
                    if ((mab[k - 1] >> (8 + k - 1)) & 1u) {
                        const int L = lab[k - 1];
                        multi |= cand != kInf && L != cand;
                        cand = min(cand, L);
                    }
                } else {
                    // from a row of the band above: plain union, unless lane l-1 has the
                    // same edge and both rows join l-1 to l
                    const int ia = ((r - k) << s.sh) + c;
                    const bool e = inw && ((sm.mask[ia] >> (8 + k - 1)) & 1u);
                    const unsigned em = __ballot_sync(kFull, e);
                    const unsigned mb = sm.hmask[((r - k) << segs_log2) + seg];
                    const unsigned implied = (em & m & mb) << 1;
                    if (e && !((implied >> lane) & 1u)) unite(par, ia, i, s);
                }
            }
            const unsigned hasm = __ballot_sync(kFull, cand != kInf);
            int mylab = va ? sidx : -1;
            if (hasm) {
                const int X = __shfl_sync(kFull, cand, __ffs(hasm) - 1);
                const unsigned uni = __ballot_sync(kFull, !multi && (cand == kInf || cand == X));
                if (uni == kFull) {
                    if (va && (hasm & runbits)) {
                        mylab = X;
                        if (lane == st) {
                            const int old = atomicMin(par + sidx, X);
                            if (old != sidx && old != X) unite(par, old, X, s);
                        } else {
                            par[i] = X;  // shortcut for the compression pass
                        }
                    }
                } else {
                    // several labels meet: one union per distinct (run, label) pair and
                    // offset
#pragma unroll
                    for (int k = 1; k <= S; ++k) {
                        if (r - k < r0) break;
                        const int ck = ((mab[k - 1] >> (8 + k - 1)) & 1u) ? lab[k - 1] : kInf;
                        const unsigned key =
                            ck == kInf ? kFull : ((unsigned)st << 16) | (unsigned)ck;
                        const unsigned grp = __match_any_sync(kFull, key);
                        if (ck != kInf && (__ffs(grp) - 1) == lane) unite(par, sidx, ck, s);
                    }
                    __syncwarp();
                    int root = 0;
                    if (va && lane == st) {
                        int budget = s.limit;
                        root = find_smem(par, sidx, budget);
                    }
                    root = __shfl_sync(kFull, root, st);
                    if (va) {
                        mylab = root;
                        if (lane != st) par[i] = root;
                    }
                }
            }

            // offsets 2..S along the row
#pragma unroll
            for (int k = 2; k <= S; ++k) {
                const int stp = __shfl_down_sync(kFull, st, k);  // run start of lane + k
                const bool e = ((mk >> (k - 1)) & 1u) && c + k < s.W;
                const bool inseg = lane + k <= 31;
                const bool e_in = e && inseg && stp != st;
                const unsigned eb = __ballot_sync(kFull, e_in);
                if (e_in) {
                    // implied by lane l-1 when l-1 ~ l and l-1+k ~ l+k by runs
                    const bool imp = lane > 0 && ((eb >> (lane - 1)) & 1u) &&
                                     ((m >> (lane - 1)) & 1u) && ((m >> (lane + k - 1)) & 1u);
                    if (!imp) unite(par, sidx, base + stp, s);
                } else if (e && !inseg) {
                    // into the next segment: covered when this run reaches lane 31, joins
                    // lane 0 of the next segment, and the target lies in that first run
                    const int t = lane + k - 32;
                    const unsigned mn = sm.hmask[u + 1];
                    const unsigned need_bits = (1u << t) - 1u;
                    const bool joined = en == 31 && ((m >> 31) & 1u) && ((mn & need_bits) == need_bits);
                    if (!joined) unite(par, i, i + k, s);
                }
            }
            // offset-1 link from lane 31 into the next segment (h1 implies c + 1 < W)
            if (lane == 31 && ((m >> 31) & 1u)) unite(par, i, i + 1, s);

#pragma unroll
            for (int k = S - 1; k > 0; --k) {
                lab[k] = lab[k - 1];
                mab[k] = mab[k - 1];
            }
            lab[0] = mylab;
            mab[0] = mk;
        }
    }
}

// Stage the strip and its halo into shared memory and compute the edge masks.
__device__ void phase1_edges(const Strip& s, const Carve& sm, uint64_t* bar, uint32_t parity) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;

    // 0. staging
    if (s.bulk) {
        if (warp == 0) {
            // the previous item used this memory through ordinary loads and stores
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(s.R * s.W * 4));
            __syncwarp();
            for (int r = lane; r < s.R; r += 32)
                bulk_copy_g2s(sm.stage + r * s.RP, s.range + (size_t)r * s.C + s.c0,
                              (uint32_t)(s.W * 4), bar);
        }
    } else {
        for (int r = warp; r < s.R; r += nwarps)
            for (int c = lane; c < s.W; c += 32)
                sm.stage[r * s.RP + c] = __ldg(s.range + (size_t)r * s.C + s.c0 + c);
    }
    // halo: S columns right of the strip (wrapping at the seam; 0 past the last column)
    for (int t = threadIdx.x; t < s.R * s.S; t += blockDim.x) {
        const int r = t / s.S;
        const int j = t - r * s.S;
        int col = s.c0 + s.W + j;
        float v = 0.0f;
        if (col >= s.C && s.wrap) col %= s.C;
        if (col < s.C) v = __ldg(s.range + (size_t)r * s.C + col);
        sm.stage[r * s.RP + s.W + j] = v;
    }
    if (s.bulk) {
        if (!mbar_wait(bar, parity, 1 << 22)) {
            report_timeout(s.status);
            mbar_wait(bar, parity, 1 << 22);  // let the copies in flight land
        }
    }
    __syncthreads();

    // 1. edge bits of every pixel, from shared memory
    for (int r = warp; r < s.R; r += nwarps) {
        float kh[kMaxSkip], kv[kMaxSkip];
#pragma unroll
        for (int k = 0; k < kMaxSkip; ++k) {
            kh[k] = k < s.S ? __ldg(s.kh + r * s.S + k) : 0.0f;
            kv[k] = k < s.S ? __ldg(s.kv + r * s.S + k) : 0.0f;
        }
        const float* row = sm.stage + r * s.RP;
        for (int cs = 0; cs < s.W; cs += 32) {  // same trip count on every lane
            const int c = cs + lane;
            const float a = c < s.W ? row[c] : 0.0f;
            const bool va = valid_range(a);
            unsigned m = 0;
            if (va) {
#pragma unroll
                for (int k = 1; k <= kMaxSkip; ++k) {
                    if (k > s.S) break;
                    const float b = row[c + k];
                    if (valid_range(b) && edge_pred(a, b, kh[k - 1], s.delta2)) m |= 1u << (k - 1);
                    if (r + k < s.R) {
                        const float d = row[c + k * s.RP];
                        if (valid_range(d) && edge_pred(a, d, kv[k - 1], s.delta2))
                            m |= 1u << (8 + k - 1);
                    }
                }
            }
            const unsigned vm = __ballot_sync(kFull, va);
            if (c < s.W) sm.mask[(r << s.sh) + c] = (uint16_t)m;
            if (lane == 0) sm.vmask[(r << (s.sh - 5)) + (cs >> 5)] = vm;
        }
    }
    __syncthreads();
}

__device__ void phase1_local(const Strip& s, const Carve& sm) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int segs_log2 = s.sh - 5;
    const int nunits = s.R << segs_log2;
    int* par = sm.par;
    unsigned* hmask = sm.hmask;

    // a. runs of horizontally joined pixels become stars
    for (int u = warp; u < nunits; u += nwarps) {
        const int r = u >> segs_log2;
        const int seg = u & ((1 << segs_log2) - 1);
        const int c = (seg << 5) + lane;
        const unsigned mk = c < s.W ? sm.mask[(r << s.sh) + c] : 0u;
        const bool h1 = (mk & 1u) && c + 1 < s.W;
        const unsigned m = __ballot_sync(kFull, h1);
        if (lane == 0) hmask[u] = m;
        // first lane of this lane's run: one past the highest missing link below it
        const unsigned below = ~m & ((1u << lane) - 1u);
        const int start = below ? 32 - __clz(below) : 0;
        // (validity words of segments that lie wholly past the strip width are never
        //  written; every lane there has c >= W)
        const bool va = c < s.W && ((sm.vmask[u] >> lane) & 1u);
        par[(r << s.sh) + c] = va ? (r << s.sh) + (seg << 5) + start : -1;
    }
    __syncthreads();

    switch (s.S) {
        case 1: phase1_bands<1>(s, sm); break;
        case 2: phase1_bands<2>(s, sm); break;
        case 3: phase1_bands<3>(s, sm); break;
        case 4: phase1_bands<4>(s, sm); break;
        case 5: phase1_bands<5>(s, sm); break;
        case 6: phase1_bands<6>(s, sm); break;
        case 7: phase1_bands<7>(s, sm); break;
        default: phase1_bands<8>(s, sm); break;
    }
    __syncthreads();

    // c. compress by pointer jumping: every round replaces each parent by its parent's
    //    parent; each entry has exactly one writer (its owner thread), so a round never
    //    stores a stale value over a newer one, and ceil(log2(depth)) rounds reach the roots
    {
        volatile int* vp = par;
        const int n = s.R << s.sh;
        int rounds = 0;
        bool changed = true;
        while (changed) {
            bool any = false;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int p = vp[i];
                if (p >= 0) {
                    const int gp = vp[p];
                    if (gp != p) {
                        vp[i] = gp;
                        any = true;
                    }
                }
            }
            changed = __syncthreads_or(any) != 0;
            if (++rounds > 40) {  // depth < 2^16: 17 rounds suffice
                if (threadIdx.x == 0) report_timeout(s.status);
                break;
            }
        }
    }

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
}

__device__ void phase2_merge(const Strip& s, const Carve& sm) {
    if (!s.border) return;
    const int first = s.W - s.S > 0 ? s.W - s.S : 0;
    const int ncols = s.W - first;
    const int n = s.R * ncols;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int r = t / ncols;
        const int c = first + (t - r * ncols);
        const unsigned mk = sm.mask[(r << s.sh) + c];
        for (int k = s.W - c; k <= s.S; ++k) {  // offsets that leave the strip
            if (!((mk >> (k - 1)) & 1u)) continue;
            int tc = s.c0 + c + k;
            if (tc >= s.C) tc %= s.C;  // a set bit past the last column implies wrap
            const int ga = global_of(s, sm.par[(r << s.sh) + c]);
            const int gb = __ldcg(s.labels + (size_t)r * s.C + tc);
            int budget = s.limit;
            union_global(s.labels, ga, gb, budget);
            if (budget <= 0) report_timeout(s.status);
        }
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
    __shared__ __align__(8) uint64_t tma_bar;
    if (threadIdx.x == 0) mbar_init(&tma_bar, 1);
    __syncthreads();
    uint32_t parity = 0;

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
            s.RP = (s.W + s.S + 3) & ~3;
            s.bulk = ((s.C & 3) == 0) && ((s.c0 & 3) == 0) && ((s.W & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(s.range) & 15) == 0);
            s.limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
        }
        const Carve sm = carve(smem_raw, s);

        if (active) {
            phase1_edges(s, sm, &tma_bar, parity);
            if (s.bulk) parity ^= 1u;
            phase1_local(s, sm);
        }
        __threadfence();
        cluster_barrier();
        if (active) phase2_merge(s, sm);
        __threadfence();
        cluster_barrier();
        if (active) phase3_flatten(s, sm.par);
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
