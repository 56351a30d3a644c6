// flic_label.cu — the FLIC neighbour test and connected-component labelling on sm_103a.
//
// One persistent kernel drains a queue of tasks.  A frame is split into full-height
// column strips; each strip gives two tasks.
//
//   P1 (one block, one strip; edge test + tile-local union in shared memory)
//      0. the strip's range readings, plus S halo columns on the right (wrapping to
//         column 0 at the seam), are staged into shared memory: one TMA bulk copy
//         (cp.async.bulk) per row completing on an mbarrier, or plain loads when the
//         frame is not 16-byte aligned;
//      1. every pixel's 2S edge bits (Eq. 2/3; offsets 1..S right and down, the Map
//         Connections of §III-B-2) are computed from shared memory into a 16-bit mask
//         per pixel; the staged readings are dead afterwards and their space becomes
//         the parent array;
//      a. each warp takes a 32-column row segment; the offset-1 right bits of the
//         segment are gathered with __ballot_sync and every pixel's parent is set to
//         the first pixel of its run, so a run of joined pixels becomes one star
//         without a single atomic;
//      b. bands of rows are walked top-down with the labels of the rows above in
//         registers (phase1_bands below): runs hook under the label they touch, and
//         only where labels meet is a union-find union made (__match_any_sync dedupe,
//         shared-memory atomicMin hooking to the smaller index);
//      c. segment seams: edges that cross a 32-column segment border inside the strip;
//      d. every pixel's label is written as the global index of its strip-local root (a
//         read-only walk up its short path), the minimum index of its strip-local
//         component.
//         A root's own entry is itself, so the labels buffer now holds a forest of
//         depth one per strip: the cross-strip forest needs no other memory.
//      The block that completes the last P1 task of a frame (atomic counter, fenced)
//      then runs the frame's boundary merge:
//   P2 (one block per frame; global memory): every edge that leaves a strip on the
//      right (offsets 1..S, including the azimuth wrap from the last column to the
//      first) unites the two strip-local roots with atomicMin hooking and path halving;
//      rows that ask for the same pair of roots are merged in the warp first.  The
//      block then raises the frame's ready flag.
//   P3 (one block, one strip; flatten): waits for the frame's ready flag, then every
//      pixel whose strip-local root was hooked by P2 gets the root of its tree (a
//      read-only find): label = minimum linear index of the component; -1 stays -1.
//
// P3 tasks of a frame are queued about one wave of blocks after its P1 tasks, so they
// seldom wait.  A block only ever waits for tasks that running blocks have already
// taken and that never wait themselves, so the queue cannot deadlock; the wait is
// bounded all the same and reports exhaustion in the frame's status word, as does every
// union and find loop.  The last block to leave resets the queue's counters for the next
// launch.  The labels buffer is the only global working memory besides those counters.
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

// Hook the run whose first pixel is `root` (a root, or hooked by this row already) under
// label x < root: one atomicMin; if the pixel was already hooked elsewhere (old), the
// two sets are united (the union-find retry step).
__device__ __forceinline__ void hook(int* par, int root, int x, const Strip& s) {
    const int old = atomicMin(par + root, x);
    if (old != root && old != x) unite(par, old, x, s);
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
                } else if (inw) {
                    // from a row of the band above (another warp): the upper pixel's
                    // current parent is a member of its set, so it serves as its label
                    const int ia = ((r - k) << s.sh) + c;
                    if ((sm.mask[ia] >> (8 + k - 1)) & 1u) {
                        const int L = ((volatile int*)par)[ia];
                        multi |= cand != kInf && L != cand;
                        cand = min(cand, L);
                    }
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
                            hook(par, sidx, X, s);
                        } else {
                            par[i] = X;  // shortcut for the final walk to the root
                        }
                    }
                } else {
                    // several labels meet.  Lanes are grouped by (run, label); each group's
                    // first lane hooks the run's first pixel under the label with one
                    // atomicMin, and only a hook that finds the pixel already hooked
                    // elsewhere unites the two labels.  A lane with several different
                    // labels above takes them one offset at a time.
                    const unsigned anymulti = __ballot_sync(kFull, multi);
                    if (!anymulti) {
                        const unsigned key =
                            cand == kInf ? kFull : ((unsigned)st << 16) | (unsigned)cand;
                        const unsigned grp = __match_any_sync(kFull, key);
                        if (cand != kInf && (__ffs(grp) - 1) == lane) hook(par, sidx, cand, s);
                    } else {
#pragma unroll
                        for (int k = 1; k <= S; ++k) {
                            if (r - k < 0) break;
                            int ck = kInf;
                            if (r - k >= r0) {
                                if ((mab[k - 1] >> (8 + k - 1)) & 1u) ck = lab[k - 1];
                            } else if (inw) {
                                const int ia = ((r - k) << s.sh) + c;
                                if ((sm.mask[ia] >> (8 + k - 1)) & 1u)
                                    ck = ((volatile int*)par)[ia];
                            }
                            const unsigned key =
                                ck == kInf ? kFull : ((unsigned)st << 16) | (unsigned)ck;
                            const unsigned grp = __match_any_sync(kFull, key);
                            if (ck != kInf && (__ffs(grp) - 1) == lane) hook(par, sidx, ck, s);
                        }
                    }
                    __syncwarp();
                    // the run's label: whatever its first pixel now points to
                    const int lbl = (va && lane == st) ? ((volatile int*)par)[sidx] : 0;
                    const int runlab = __shfl_sync(kFull, lbl, st);
                    if (va) {
                        mylab = runlab;
                        if (lane != st) par[i] = runlab;
                    }
                }
            }

            // offsets 2..S along the row, inside the segment (edges into the next
            // segment are left to the seam pass); nothing to do when both runs already
            // carry the same label
#pragma unroll
            for (int k = 2; k <= S; ++k) {
                const int stp = __shfl_down_sync(kFull, st, k);      // run start of lane + k
                const int labp = __shfl_down_sync(kFull, mylab, k);  // its label
                const bool e_in = ((mk >> (k - 1)) & 1u) && c + k < s.W && lane + k <= 31 &&
                                  stp != st && labp != mylab;
                const unsigned eb = __ballot_sync(kFull, e_in);
                if (e_in) {
                    // implied by lane l-1 when l-1 ~ l and l-1+k ~ l+k by runs
                    const bool imp = lane > 0 && ((eb >> (lane - 1)) & 1u) &&
                                     ((m >> (lane - 1)) & 1u) && ((m >> (lane + k - 1)) & 1u);
                    if (!imp) unite(par, sidx, base + stp, s);
                }
            }

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

// Edges that cross a 32-column segment border inside the strip (offsets 1..S to the
// right), after the band pass.  Lanes are rows; the pair to unite is the current parents
// of the two ends, and of consecutive rows asking for the same pair only the first asks.
__device__ void phase1_seams(const Strip& s, const Carve& sm) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    volatile int* vp = sm.par;
    const int nborders = (s.W - 1) >> 5;  // segment borders g | g+1 with (g+1)*32 < W
    const int rblocks = (s.R + 31) >> 5;
    for (int job = warp; job < nborders * rblocks; job += nwarps) {
        const int g = job / rblocks;
        const int r = ((job - g * rblocks) << 5) + lane;
        const bool row_ok = r < s.R;
        const int cb = (g + 1) << 5;  // first column of the next segment
        int done_a = -1, done_b = -1;  // the last pair this lane united
        for (int c = cb - s.S; c < cb; ++c) {
            const unsigned mk = row_ok ? sm.mask[(r << s.sh) + c] : 0u;
            for (int k = cb - c; k <= s.S; ++k) {
                const bool e = ((mk >> (k - 1)) & 1u) && c + k < s.W;
                int a = 0, b = 0;
                if (e) {
                    a = vp[(r << s.sh) + c];
                    b = vp[(r << s.sh) + c + k];
                }
                const int pa = __shfl_up_sync(kFull, a, 1);
                const int pb = __shfl_up_sync(kFull, b, 1);
                const unsigned em = __ballot_sync(kFull, e);
                const bool dup = (lane > 0 && ((em >> (lane - 1)) & 1u) && pa == a && pb == b) ||
                                 (a == done_a && b == done_b);
                if (e && !dup && a != b) {
                    unite(sm.par, a, b, s);
                    done_a = a;
                    done_b = b;
                }
            }
        }
    }
}

// Edge bits of every pixel from the staged readings: bit k-1 = edge to the pixel k
// columns right (into the halo at the strip's right edge), bit 8+k-1 = edge to the pixel
// k rows down; validity as one ballot word per 32-column segment.
template <int S>
__device__ void mask_rows(const Strip& s, const Carve& sm) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int r = warp; r < s.R; r += nwarps) {
        float kh[S], kv[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            kh[k] = __ldg(s.kh + r * S + k);
            kv[k] = __ldg(s.kv + r * S + k);
        }
        const int down = min(S, s.R - 1 - r);  // vertical offsets that stay in the frame
        const float* row = sm.stage + r * s.RP;
        for (int cs = 0; cs < s.W; cs += 32) {  // same trip count on every lane
            const int c = cs + lane;
            const float a = c < s.W ? row[c] : 0.0f;
            const bool va = valid_range(a);
            unsigned m = 0;
            if (va) {
                // with a valid, a neighbour b is a measurement iff b > 0: +inf and NaN
                // fail d2 <= delta2 by themselves
#pragma unroll
                for (int k = 1; k <= S; ++k) {
                    const float b = row[c + k];
                    const float d = k <= down ? row[c + k * s.RP] : 0.0f;
                    float dh, dv;
                    edge_d2_pair(a, b, d, kh[k - 1], kv[k - 1], dh, dv);
                    if (b > 0.0f && dh <= s.delta2) m |= 1u << (k - 1);
                    if (d > 0.0f && dv <= s.delta2) m |= 1u << (8 + k - 1);
                }
            }
            const unsigned vm = __ballot_sync(kFull, va);
            if (c < s.W) sm.mask[(r << s.sh) + c] = (uint16_t)m;
            if (lane == 0) sm.vmask[(r << (s.sh - 5)) + (cs >> 5)] = vm;
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
    switch (s.S) {
        case 1: mask_rows<1>(s, sm); break;
        case 2: mask_rows<2>(s, sm); break;
        case 3: mask_rows<3>(s, sm); break;
        case 4: mask_rows<4>(s, sm); break;
        case 5: mask_rows<5>(s, sm); break;
        case 6: mask_rows<6>(s, sm); break;
        case 7: mask_rows<7>(s, sm); break;
        default: mask_rows<8>(s, sm); break;
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
    phase1_seams(s, sm);
    __syncthreads();

    // c/d. every pixel's label: the global index of its strip-local root
    {
        const volatile int* vp = par;
        int last_p = -1, last_root = -1;
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
                    int p = c + q < s.W ? vp[base + c + q] : -1;
                    if (p >= 0) {
                        // read-only walk to the strip-local root (paths are short after the
                        // band pass; nothing writes par any more); neighbours usually share
                        // their parent, so the last walk is remembered
                        if (p != last_p) {
                            int budget = s.limit;
                            last_root = global_of(s, find_smem_ro(vp, p, budget));
                            if (budget <= 0) report_timeout(s.status);
                            last_p = p;
                        }
                        v[q] = last_root;
                    } else {
                        v[q] = -1;
                    }
                }
                if (vec && c + 4 <= s.W) {
                    __stcg(reinterpret_cast<int4*>(out + c), make_int4(v[0], v[1], v[2], v[3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c + q < s.W) __stcg(out + c + q, v[q]);
                }
            }
        }
    }
}

// P2: the boundary merge of one border (strip b's right edge, to strip b + 1 or across
// the seam to strip 0), by the block that completes the second of its two strips.  Lanes
// are rows; each lane loads its row's S readings and labels on both sides of the border
// at once, tests the crossing edges, and of consecutive rows that would unite the same
// pair of strip-local roots only the first asks.
__device__ __forceinline__ unsigned long long volatile_load_u64(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

template <int S>
__device__ void border_merge_s(const FrameDesc& f, int b, int limit,
                               unsigned long long* pair_set) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int R = f.rows, C = f.cols;
    const int c0 = b * f.strip_w;
    const int W = min(f.strip_w, C - c0);  // >= S (several strips, or C >= S)
    const int first = W - S;
    const int rblocks = (R + 31) >> 5;
    for (int rb = warp; rb < rblocks; rb += nwarps) {
        const int r = (rb << 5) + lane;
        const bool row_ok = r < R;
        const float* rrow = f.range + (size_t)(row_ok ? r : 0) * C;
        const int32_t* lrow = f.labels + (size_t)(row_ok ? r : 0) * C;
        float av[S], dv[S], kh[S];
        int la[S], lb[S];
        int done_a = -1, done_b = -1;  // the last pair this lane united
#pragma unroll
        for (int j = 0; j < S; ++j) {
            int tc = c0 + W + j;  // j-th column past the border
            if (tc >= C && f.wrap) tc %= C;
            const bool tok = row_ok && tc < C;
            av[j] = row_ok ? load_range(rrow + c0 + first + j) : 0.0f;
            la[j] = row_ok ? __ldcg(lrow + c0 + first + j) : 0;
            dv[j] = tok ? load_range(rrow + tc) : 0.0f;
            lb[j] = tok ? __ldcg(lrow + tc) : 0;
            kh[j] = __ldg(f.kh + (row_ok ? r : 0) * S + j);
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {            // source column first + j
#pragma unroll
            for (int k = S - j; k <= S; ++k) {   // offsets that cross: target j + k - S
                const int t = j + k - S;
                const bool e = av[j] > 0.0f && dv[t] > 0.0f && edge_pred(av[j], dv[t], kh[k - 1], f.delta2);
                const int ga = la[j], gb = lb[t];
                const int pa = __shfl_up_sync(kFull, ga, 1);
                const int pb = __shfl_up_sync(kFull, gb, 1);
                const unsigned em = __ballot_sync(kFull, e);
                // dropped when the row above asks for the same pair, or when this row
                // already asked for it at another column or offset
                const bool dup = (lane > 0 && ((em >> (lane - 1)) & 1u) && pa == ga && pb == gb) ||
                                 (ga == done_a && gb == done_b);
                if (e && !dup && ga != gb) {
                    // the other warps of this block may have united this pair already
                    const unsigned long long key =
                        ((unsigned long long)(unsigned)ga << 32) | (unsigned)gb;
                    const int h = (int)((key * 0x9E3779B97F4A7C15ull) >> 58);  // 64 entries
                    if (volatile_load_u64(pair_set + h) != key) {
                        int budget = limit;
                        union_global(f.labels, ga, gb, budget);
                        if (budget <= 0) report_timeout(f.status);
                        pair_set[h] = key;
                    }
                    done_a = ga;
                    done_b = gb;
                }
            }
        }
    }
}

// The same for a single strip narrower than S (wrapping onto itself): plain loops.
__device__ void border_merge_narrow(const FrameDesc& f, int limit) {
    const int R = f.rows, C = f.cols, S = f.skip;
    for (int t = threadIdx.x; t < R * C; t += blockDim.x) {
        const int r = t / C, c = t - r * C;
        const float a = load_range(f.range + t);
        if (!(a > 0.0f)) continue;
        for (int k = C - c; k <= S; ++k) {
            const int tc = (c + k) % C;
            const float d = load_range(f.range + (size_t)r * C + tc);
            if (d > 0.0f && edge_pred(a, d, __ldg(f.kh + r * S + k - 1), f.delta2)) {
                int budget = limit;
                union_global(f.labels, __ldcg(f.labels + t), __ldcg(f.labels + (size_t)r * C + tc),
                             budget);
                if (budget <= 0) report_timeout(f.status);
            }
        }
    }
}

__device__ void border_merge(const FrameDesc& f, int b) {
    const int limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
    // root pairs this block has united during this merge (a cache: a collision only
    // costs a repeated union)
    __shared__ unsigned long long pair_set[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) pair_set[i] = ~0ull;
    __syncthreads();
    const int W = min(f.strip_w, f.cols - b * f.strip_w);
    if (W < f.skip) {
        border_merge_narrow(f, limit);
        return;
    }
    switch (f.skip) {
        case 1: border_merge_s<1>(f, b, limit, pair_set); break;
        case 2: border_merge_s<2>(f, b, limit, pair_set); break;
        case 3: border_merge_s<3>(f, b, limit, pair_set); break;
        case 4: border_merge_s<4>(f, b, limit, pair_set); break;
        case 5: border_merge_s<5>(f, b, limit, pair_set); break;
        case 6: border_merge_s<6>(f, b, limit, pair_set); break;
        case 7: border_merge_s<7>(f, b, limit, pair_set); break;
        default: border_merge_s<8>(f, b, limit, pair_set); break;
    }
}

// P3: flatten one strip once its frame's forest is final.  Consecutive pixels usually
// share a strip-local root, so each thread remembers its last lookup.
__device__ void phase3_strip(const FrameDesc& f, int si) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int c0 = si * f.strip_w;
    const int W = min(f.strip_w, f.cols - c0);
    const int limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
    const bool vec = ((f.cols & 3) == 0) && ((c0 & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(f.labels) & 15) == 0);
    int last_l = -1, last_root = -1;
    for (int r = warp; r < f.rows; r += nwarps) {
        int32_t* row = f.labels + (size_t)r * f.cols + c0;
        for (int c = lane * 4; c < W; c += 128) {
            int v[4];
            const bool full = vec && c + 4 <= W;
            if (full) {
                const int4 x = __ldcg(reinterpret_cast<const int4*>(row + c));
                v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = c + q < W ? __ldcg(row + c + q) : -1;
            }
            bool changed = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int l = v[q];
                if (l < 0) continue;
                if (l != last_l) {
                    int budget = limit;
                    last_root = find_global(f.labels, l, budget, false);
                    if (budget <= 0) report_timeout(f.status);
                    last_l = l;
                }
                if (last_root != l) {
                    v[q] = last_root;
                    changed = true;
                }
            }
            if (changed) {
                if (full) {
                    __stcg(reinterpret_cast<int4*>(row + c), make_int4(v[0], v[1], v[2], v[3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c + q < W) __stcg(row + c + q, v[q]);
                }
            }
        }
    }
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(512, 2) flic_label_kernel(const LabelLaunch L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t tma_bar;
    __shared__ int task_sh;
    __shared__ int flag_sh;
    if (threadIdx.x == 0) mbar_init(&tma_bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    const int ntasks = L.dims ? L.dims[0] : L.ntasks;
    const int nframes = L.dims ? L.dims[1] : L.nframes;

    while (true) {
        if (threadIdx.x == 0) task_sh = atomicAdd(L.counters + kCtrNext, 1);
        __syncthreads();
        const int t = task_sh;
        __syncthreads();  // task_sh is rewritten by the next iteration
        if (t >= ntasks) break;

        int fi, si, kind;
        if (L.tasks) {
            const Task tk = L.tasks[t];
            fi = tk.frame;
            si = tk.strip;
            kind = tk.kind;
        } else {  // one frame: P1 of strips 0..n-1, then P3 of strips 0..n-1
            fi = 0;
            si = t < L.single.nstrips ? t : t - L.single.nstrips;
            kind = t < L.single.nstrips ? kTaskP1 : kTaskP3;
        }
        const FrameDesc f = L.frames ? L.frames[fi] : L.single;
        const bool border = f.nstrips > 1 || f.wrap;
        // [borders merged, ready, arrivals at border 0, 1, ...]
        int* done_ctr = L.counters + kCtrFrames + kCtrPerFrame * fi;

        if (kind == kTaskP1) {
            Strip s{};
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
            s.border = border;
            s.c0 = si * f.strip_w;
            s.W = min(f.strip_w, s.C - s.c0);
            s.sh = f.pitch_log2;
            s.RP = (s.W + s.S + 3) & ~3;
            s.bulk = ((s.C & 3) == 0) && ((s.c0 & 3) == 0) && ((s.W & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(s.range) & 15) == 0);
            s.limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
            const Carve sm = carve(smem_raw, s);
            phase1_edges(s, sm, &tma_bar, parity);
            if (s.bulk) parity ^= 1u;
            phase1_local(s, sm);
            if (border) {
                // arrive at the (up to two) borders of this strip; the second arrival at a
                // border merges it, and the last merged border makes the frame ready
                const int n = f.nstrips;
                const int nb = f.wrap ? n : n - 1;
                __threadfence();
                __syncthreads();
                for (int side = 0; side < 2; ++side) {
                    const int b = side == 0 ? si : si - 1;  // right border, then left border
                    const int bb = b < 0 ? (f.wrap ? n - 1 : -1) : b;
                    if (bb < 0 || bb >= nb || (side == 1 && n == 1)) continue;  // uniform
                    if (threadIdx.x == 0) {
                        const int need = n == 1 ? 1 : 2;
                        flag_sh = atomicAdd(done_ctr + 2 + bb, 1) == need - 1;
                    }
                    __syncthreads();
                    if (flag_sh) {
                        __threadfence();
                        border_merge(f, bb);
                        __threadfence();
                        __syncthreads();
                        if (threadIdx.x == 0 && atomicAdd(done_ctr, 1) == nb - 1)
                            st_release(done_ctr + 1, 1);
                    }
                    __syncthreads();
                }
            }
        } else {
            if (threadIdx.x == 0) {
                int it = 0;
                flag_sh = 1;
                while (ld_acquire(done_ctr + 1) == 0) {
                    __nanosleep(128);
                    if (++it > (1 << 24)) {  // ~2 s: give up and leave the strip alone,
                        report_timeout(f.status);  // its labels may not be written yet
                        flag_sh = 0;
                        break;
                    }
                }
            }
            __syncthreads();
            if (flag_sh) phase3_strip(f, si);
        }
        __syncthreads();  // shared memory is reused by the next task
    }

    // the last block to leave resets the counters for the next launch on this stream
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(L.counters + kCtrExit, 1) == (int)gridDim.x - 1) {
            for (size_t i = 0; i < counter_ints(nframes); ++i) L.counters[i] = 0;
            __threadfence();
        }
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
    return cudaFuncSetAttribute(flic_label_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)max_smem);
}

cudaError_t launch_label(const LabelLaunch& L, int grid, int threads, size_t smem,
                         cudaStream_t stream) {
    flic_label_kernel<<<grid, threads, smem, stream>>>(L);
    return cudaGetLastError();
}

cudaError_t label_blocks_per_sm(int threads, size_t smem, int* out) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, flic_label_kernel, threads, smem);
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
