// flic_label.cu — the FLIC neighbour test and connected-component labelling on sm_103a.
//
// One persistent kernel drains a queue of tasks.  A frame is split into full-height
// column strips; each strip gives two tasks.
//
//   P1 (one block, one strip; edge test + tile-local union in shared memory)
//      0. the strip's range readings are staged into shared memory: one TMA bulk copy
//         (cp.async.bulk) per row completing on an mbarrier, or plain loads when the
//         frame is not 16-byte aligned;
//      1. every pixel's 2S edge bits (Eq. 2/3; offsets 1..S right and down, the Map
//         Connections of section III-B-2) are computed from shared memory, lanes =
//         columns, and gathered with __ballot_sync into 32-bit words per 32-column row
//         segment: one word of measurements, one per right offset, one per down offset.
//         The staged readings are dead afterwards and their space becomes the parent
//         array.  Edges that leave the strip are not recorded (P2 tests them again);
//      a. from here one thread owns one row segment and works on whole words.  A run of
//         pixels joined by offset-1 right edges is one union-find node, its first pixel
//         (run starts = measurements without a right edge from the left neighbour).  The
//         other edges give pairs of runs: of all edges joining the same two runs only the
//         first is taken (the words are cut at the run starts of both ends), and an edge
//         of offset k >= 2 that two shorter edges through one pixel already imply is
//         dropped — on smooth surfaces nearly all of them;
//      b. every run start is linked to the smallest run its pairs reach (one shared-
//         memory atomicMin per pair, no finds), which builds most of the forest;
//      c. every pair is united (finds with path halving, atomicMin hooking of the larger
//         root under the smaller, retry when a hook loses a race);
//      d. every run start's entry is set to its root;
//      e. every pixel's label is written as the global index of its run's strip-local
//         root, the minimum index of its strip-local component.
//         A root's own entry is itself, so the labels buffer now holds a forest of
//         depth one per strip: the cross-strip forest needs no other memory.
//      A strip then arrives at its (up to two) borders; the block that arrives second
//      at a border merges it:
//   P2 (one block, one border; global memory): every edge that crosses the border to
//      the right (offsets 1..S, including the azimuth wrap from the last column to the
//      first) unites the two strip-local roots with atomicMin hooking and path halving;
//      rows that ask for the same pair of roots are merged in the warp first.  Each
//      merged border is counted (a release reduction); the frame is ready when the
//      count reaches its number of borders.
//   P3 (one block, one strip; flatten): waits until its frame is ready, then every
//      pixel whose strip-local root was hooked by P2 gets the root of its tree (a
//      read-only find): label = minimum linear index of the component; -1 stays -1.
//
// P3 tasks of a frame are queued a few waves of blocks after its P1 tasks, so they
// seldom wait.  A block only ever waits for tasks that come before its own in the queue,
// which running blocks have already taken and which never wait themselves, so the queue
// cannot deadlock; the wait is bounded all the same and reports exhaustion in the
// frame's status word, as does every union and find loop.  The last block to leave resets the queue's counters for the next
// launch.  The labels buffer is the only global working memory besides those counters.
#include <algorithm>
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
    const float* kd;   // diagonal constants, nullptr: no diagonal Map Connections
    int32_t* status;
    int R, C, S;
    float delta2;
    bool wrap;
    bool lattice;  // sparse Map Connection (FrameDesc::lattice)
    int c0, W;     // first column and width of the strip
    int sh;        // local pitch = 1 << sh (>= 32, >= W)
    int RP;        // row pitch of the staged readings (>= W + S, multiple of 4)
    bool bulk;     // rows are 16-byte aligned: stage with TMA bulk copies
    int limit;
    const float* gnd;  // ground table, nullptr: no ground extraction
    float gnd_tan, gnd_height;
};

// Shared-memory carve-up of one strip (byte offsets; see strip_smem_bytes on the host).
struct Carve {
    float* stage;      // R x RP staged readings; reused as the parent array (R x P)
    int* par;
    unsigned* words;   // R x P/32 row segments x (2S + 1) ballot words
    unsigned* dwords;  // the same for the diagonal Map Connections (when there are any)
};

__device__ __forceinline__ Carve carve(unsigned char* base, const Strip& s) {
    Carve c;
    const int P = 1 << s.sh;
    const int a_words = s.R * (s.RP > P ? s.RP : P);
    c.stage = reinterpret_cast<float*>(base);
    c.par = reinterpret_cast<int*>(base);
    c.words = reinterpret_cast<unsigned*>(base + 4 * (size_t)a_words);
    c.dwords = c.words + (size_t)(s.R << (s.sh - 5)) * (2 * s.S + 1);
    return c;
}

__device__ __forceinline__ int global_of(const Strip& s, int local) {
    return (local >> s.sh) * s.C + s.c0 + (local & ((1 << s.sh) - 1));
}

// ---- word helpers ------------------------------------------------------------------------

// The ballot words of a strip.  Row segment u = r * P/32 + seg covers local pixels
// 32u .. 32u + 31 and owns the 2S + 1 consecutive words w[u * (2S + 1) + p]: [0] the pixel
// is a measurement, [k] edge to the pixel k columns right, [S + k] edge to the pixel k
// rows down (k = 1..S).  Bit j is column 32 seg + j.  The stride 2S + 1 is odd, so 32
// threads reading the same word of 32 consecutive segments hit 32 different banks.
template <int S>
struct Words {
    static constexpr int NP = 2 * S + 1;
    unsigned* w;
    int n;  // row segments
    __device__ __forceinline__ unsigned operator()(int p, int u) const { return w[u * NP + p]; }
    // run starts: measurements that no offset-1 edge reaches from the left
    __device__ __forceinline__ unsigned starts(int u) const {
        return w[u * NP] & ~(w[u * NP + 1] << 1);
    }
};

template <int S>
__device__ __forceinline__ Words<S> words_of(const Strip& s, const Carve& sm) {
    return Words<S>{sm.words, s.R << (s.sh - 5)};
}

// The diagonal words of a strip, in the same layout: [k] edge from the pixel to the pixel
// k rows down and k columns right, [S + k] k rows down and k columns left (k = 1..S);
// [0] is unused.
template <int S>
__device__ __forceinline__ Words<S> dwords_of(const Strip& s, const Carve& sm) {
    return Words<S>{sm.dwords, s.R << (s.sh - 5)};
}

// Bits 0..c of a word (c in 0..31).
__device__ __forceinline__ unsigned upto(int c) { return (2u << c) - 1u; }

// Index of the highest set bit (x != 0).
__device__ __forceinline__ int top_bit(unsigned x) { return 31 - __clz(x); }

// x without its bits below the lowest bit of `cuts` above column c (empty if none).
__device__ __forceinline__ unsigned skip_to_next(unsigned x, unsigned cuts, int c) {
    const unsigned nb = cuts & ~upto(c);
    return x & ~((nb & (0u - nb)) - 1u);
}

// ---- the strip-local forest ----------------------------------------------------------------
// Nodes are local pixel indices (r * P + c); only run starts are ever nodes.  par[x] == x:
// root; par[x] < x otherwise (hooking always goes to the smaller index, so the root of a
// set is its minimum element).  Node x lives at slot(x): its column bits are XORed with
// the low bits of its row segment, so that the first pixels of 32 consecutive segments
// (the commonest run starts) fall into 32 different banks.

__device__ __forceinline__ int slot(int x) { return x ^ ((x >> 5) & 31); }

// Find with path halving.  A halving store racing with an atomicMin only replaces one
// ancestor by another; a union whose atomicMin lost the race retries with what it found.
__device__ __forceinline__ int find_run(volatile int* par, int x, int& budget) {
    while (true) {
        const int p = par[slot(x)];
        if (p == x) return x;
        const int gp = par[slot(p)];
        if (gp == p) return p;
        par[slot(x)] = gp;
        x = gp;
        if (--budget <= 0) return x;
    }
}

// Read-only find, once no union is running any more.
__device__ __forceinline__ int find_run_ro(const volatile int* par, int x, int& budget) {
    int p = par[slot(x)];
    while (p != x) {
        x = p;
        p = par[slot(x)];
        if (--budget <= 0) break;
    }
    return x;
}

__device__ __forceinline__ void unite(int* par, int a, int b, const Strip& s) {
    volatile int* vp = par;
    int budget = s.limit;
    while (budget > 0) {
        a = find_run(vp, a, budget);
        b = find_run(vp, b, budget);
        if (a == b) break;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(par + slot(b), a);
        if (old == b) break;
        b = old;
        --budget;
    }
    if (budget <= 0) report_timeout(s.status);
}

// 0. Stage the strip's readings into shared memory (row pitch RP).
__device__ void phase1_stage(const Strip& s, const Carve& sm, uint64_t* bar, uint32_t parity) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    if (s.bulk) {
        if (warp == 0) {
            // the previous item used this memory through ordinary loads and stores
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(s.R * s.W * 4));
            __syncwarp();
            for (int r = lane; r < s.R; r += 32)
                bulk_copy_g2s(sm.stage + r * s.RP, s.range + (size_t)r * s.C + s.c0,
                              (uint32_t)(s.W * 4), bar);
            if (!mbar_wait(bar, parity, 1 << 22)) {
                report_timeout(s.status);
                mbar_wait(bar, parity, 1 << 22);  // let the copies in flight land
            }
        }
    } else {
        for (int r = warp; r < s.R; r += nwarps)
            for (int c = lane; c < s.W; c += 32)
                sm.stage[r * s.RP + c] = __ldg(s.range + (size_t)r * s.C + s.c0 + c);
    }
    __syncthreads();
}

// 0b. Ground extraction (§III-A): readings that span a horizontal surface with the reading
//     above them become non-measurements in the staged strip, before the edge test.  All
//     decisions are taken first (ballot words, in the space the edge words take later),
//     then applied, so that no decision reads a reading already cleared.  The first row
//     decides as the second.
__device__ void phase1_ground(const Strip& s, const Carve& sm) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsl = s.sh - 5;
    unsigned* gw = sm.words;  // R x P/32 words
    for (int r = warp; r < s.R; r += nwarps) {
        const int rt = r == 0 ? 1 : r;
        const float* up = sm.stage + (rt - 1) * s.RP;
        const float* lo = sm.stage + rt * s.RP;
        const float* own = sm.stage + r * s.RP;
        for (int cs = 0; cs < s.W; cs += 32) {  // same trip count on every lane
            const int c = cs + lane;
            bool g = false;
            if (c < s.W) {
                const float d = own[c];
                if (valid_range(d)) {
                    const float d1 = up[c], d2 = lo[c];
                    g = ground_horizontal(valid_range(d1) ? d1 : 0.0f, valid_range(d2) ? d2 : 0.0f,
                                          s.gnd + rt * kGroundFields) &&
                        !ground_above_line(d, s.gnd + r * kGroundFields, s.gnd_tan, s.gnd_height);
                }
            }
            const unsigned w = __ballot_sync(kFull, g);
            if (lane == 0) gw[(r << nsl) + (cs >> 5)] = w;
        }
    }
    __syncthreads();
    for (int r = warp; r < s.R; r += nwarps) {
        float* own = sm.stage + r * s.RP;
        for (int cs = 0; cs < s.W; cs += 32) {
            const int c = cs + lane;
            if (c < s.W && ((gw[(r << nsl) + (cs >> 5)] >> lane) & 1u)) own[c] = 0.0f;
        }
    }
    __syncthreads();
}

// 0c. Every staged reading that is no measurement becomes +inf (after the ground pass,
//     which clears ground readings to 0).  A pair with such a reading then fails the edge
//     test by itself: (a - inf)^2 and K (a inf) are +inf or NaN, and so is d2.  The row
//     pitch is a multiple of 4, so the pass runs over float4s (padding included, never
//     read).
__device__ __forceinline__ float no_reading() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ float clean_reading(float x) { return x > 0.0f ? x : no_reading(); }

__device__ void phase1_clean(const Strip& s, const Carve& sm) {
    float4* st = reinterpret_cast<float4*>(sm.stage);
    const int n4 = (s.R * s.RP) >> 2;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        float4 v = st[i];
        v.x = clean_reading(v.x);
        v.y = clean_reading(v.y);
        v.z = clean_reading(v.z);
        v.w = clean_reading(v.w);
        st[i] = v;
    }
    __syncthreads();
}

// The 2S + 1 ballot words of one 32-column chunk of row `row` (lanes = columns).  An
// interior chunk has S rows below it and S columns right of it inside the strip, so it
// needs no bounds tests.  Right edges whose far end lies past the strip are left out (the
// boundary merge tests them).  The staged readings are clean (phase1_clean): a pixel is a
// measurement iff its reading is below +inf, and a pair passes the test only if both are.
template <int S, bool kInterior>
__device__ __forceinline__ void mask_chunk(const Strip& s, const float* row, int c, int down,
                                           const float (&kh)[S], const float (&kv)[S],
                                           unsigned (&w)[2 * S + 1]) {
    const bool in = kInterior || c < s.W;
    const float a = in ? row[c] : no_reading();
    w[0] = __ballot_sync(kFull, a < no_reading());
#pragma unroll
    for (int k = 1; k <= S; ++k) {
        const bool hin = kInterior || c + k < s.W;
        const bool vin = kInterior || (in && k <= down);
        const float b = hin ? row[c + k] : no_reading();
        const float d = vin ? row[c + k * s.RP] : no_reading();
        float dh, dv;
        edge_d2_pair(a, b, d, kh[k - 1], kv[k - 1], dh, dv);
        w[k] = __ballot_sync(kFull, dh <= s.delta2);
        w[S + k] = __ballot_sync(kFull, dv <= s.delta2);
    }
}

// The diagonal words of the same chunk (§III-B-2, Map Connections along the diagonals):
// edges (r, c)-(r+k, c+k) and (r, c)-(r+k, c-k) whose far end lies inside the strip (the
// boundary merge tests the others), with the constant kd of the pair's upper row.
template <int S, bool kInterior>
__device__ __forceinline__ void diag_chunk(const Strip& s, const float* row, int c, int down,
                                           const float (&kd)[S], unsigned w0,
                                           unsigned (&d)[2 * S + 1]) {
    const bool in = kInterior || c < s.W;
    const float a = in ? row[c] : no_reading();
    d[0] = 0u;
#pragma unroll
    for (int k = 1; k <= S; ++k) {
        const bool vin = kInterior || (in && k <= down);
        const bool rin = vin && (kInterior || c + k < s.W);
        const bool lin = vin && c >= k;
        const float br = rin ? row[c + k + k * s.RP] : no_reading();
        const float bl = lin ? row[c - k + k * s.RP] : no_reading();
        float dr, dl;
        edge_d2_pair(a, br, bl, kd[k - 1], kd[k - 1], dr, dl);
        d[k] = __ballot_sync(kFull, dr <= s.delta2);
        d[S + k] = __ballot_sync(kFull, dl <= s.delta2);
    }
}

// 1b. The sparse Map Connection (§III-B-2, every S-th point joined at offset S), applied to
//     the ballot words of the whole strip (one thread per row segment): offsets 2..S-1
//     dropped, offset S kept only where the row and the global column are multiples of S.
template <int S>
__device__ void lattice_words(const Strip& s, const Carve& sm) {
    if constexpr (S >= 2) {
        constexpr int NP = Words<S>::NP;
        unsigned pat = 0;  // bits 0, S, 2S, ... of a word
#pragma unroll
        for (int b = 0; b < 32; b += S) pat |= 1u << b;
        const int nsl = s.sh - 5;
        const int n = s.R << nsl;
        for (int u = threadIdx.x; u < n; u += blockDim.x) {
            unsigned* w = sm.words + (size_t)u * NP;
            const int r = u >> nsl;
            const int base = s.c0 + ((u & ((1 << nsl) - 1)) << 5);  // global column of bit 0
            const unsigned keep = r % S == 0 ? pat << ((S - base % S) % S) : 0u;
#pragma unroll
            for (int k = 2; k < S; ++k) {
                w[k] = 0u;
                w[S + k] = 0u;
            }
            w[S] &= keep;
            w[2 * S] &= keep;
        }
    }
}

// 1. The ballot words of every row segment from the staged readings (a warp per row).
template <int S, bool D>
__device__ void mask_rows(const Strip& s, const Carve& sm) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const Words<S> wd = words_of<S>(s, sm);
    const Words<S> dd = dwords_of<S>(s, sm);
    for (int r = warp; r < s.R; r += nwarps) {
        float kh[S], kv[S], kd[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            kh[k] = __ldg(s.kh + r * S + k);
            kv[k] = __ldg(s.kv + r * S + k);
            kd[k] = D ? __ldg(s.kd + r * S + k) : 0.0f;
        }
        const int down = min(S, s.R - 1 - r);  // vertical offsets that stay in the frame
        const float* row = sm.stage + r * s.RP;
        unsigned* out = wd.w + (size_t)(r << (s.sh - 5)) * Words<S>::NP;
        unsigned* dout = dd.w + (size_t)(r << (s.sh - 5)) * Words<S>::NP;
        // chunks with cs + 32 + S <= W and S rows below are interior
        const int interior = down == S && s.W >= S ? ((s.W - S) >> 5) << 5 : 0;
        int cs = 0;
        for (; cs < interior; cs += 32) {  // same trip counts on every lane
            unsigned w[2 * S + 1];
            mask_chunk<S, true>(s, row, cs + lane, down, kh, kv, w);
            // every lane stores the same word to the same address: one write
#pragma unroll
            for (int p = 0; p <= 2 * S; ++p) out[(cs >> 5) * Words<S>::NP + p] = w[p];
            if constexpr (D) {
                unsigned d[2 * S + 1];
                diag_chunk<S, true>(s, row, cs + lane, down, kd, w[0], d);
#pragma unroll
                for (int p = 0; p <= 2 * S; ++p) dout[(cs >> 5) * Words<S>::NP + p] = d[p];
            }
        }
        for (; cs < s.W; cs += 32) {
            unsigned w[2 * S + 1];
            mask_chunk<S, false>(s, row, cs + lane, down, kh, kv, w);
#pragma unroll
            for (int p = 0; p <= 2 * S; ++p) out[(cs >> 5) * Words<S>::NP + p] = w[p];
            if constexpr (D) {
                unsigned d[2 * S + 1];
                diag_chunk<S, false>(s, row, cs + lane, down, kd, w[0], d);
#pragma unroll
                for (int p = 0; p <= 2 * S; ++p) dout[(cs >> 5) * Words<S>::NP + p] = d[p];
            }
        }
    }
}

// a. Every run's first pixel becomes a root of its own (one thread per row segment).
template <int S>
__device__ void init_runs(const Strip& s, const Carve& sm) {
    const Words<S> wd = words_of<S>(s, sm);
    const int nsl = s.sh - 5;
    for (int u = threadIdx.x; u < wd.n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= s.W) continue;  // segment past the strip
        unsigned x = wd.starts(u);
        while (x) {
            const int c = (u << 5) + __ffs(x) - 1;
            x &= x - 1u;
            sm.par[slot(c)] = c;
        }
    }
}

// Every pair of runs (x, y), y < x, that an edge inside the strip joins, for the edges whose
// near end lies in row segment u: op(x, y).  Of all edges that join the same two runs only
// the first is taken — along a segment the pair of runs an offset joins only changes at a
// run start of either end, so after an edge at column c the word skips to the next such
// cut — and an edge of offset k >= 2 is dropped where two shorter edges through one pixel
// of the same column (up) or row (right) already join its ends: by induction on k those
// are taken or dropped for the same reason, so the components do not change.
template <int S, class Op>
__device__ __forceinline__ void for_each_pair(const Strip& s, const Words<S>& wd, int u, Op op) {
    const int nsl = s.sh - 5;
    const int NS = 1 << nsl;
    const int r = u >> nsl;
    const unsigned va = wd(0, u);
    if (!va) return;
    const unsigned h1 = wd(1, u);
    const unsigned rs = va & ~(h1 << 1);
    const int base = u << 5;

    // offsets 1..S up: the down word k of row r - k joins (r - k, c) and (r, c)
#pragma unroll
    for (int k = 1; k <= S; ++k) {
        if (r - k < 0) break;
        const int uu = u - k * NS;
        unsigned v = wd(S + k, uu);
        if (k >= 2)  // via (r - 1, c) or via (r - k + 1, c)
            v &= ~((wd(S + 1, u - NS) & wd(S + k - 1, uu)) |
                   (wd(S + 1, uu) & wd(S + k - 1, uu + NS)));
        if (!v) continue;
        const unsigned rsu = wd.starts(uu);
        const unsigned cuts = rs | rsu;
        const int ubase = base - (k << s.sh);
        do {
            const int c = __ffs(v) - 1;
            const unsigned m = upto(c);
            op(base + top_bit(rs & m), ubase + top_bit(rsu & m));
            v = skip_to_next(v, cuts, c);
        } while (v);
    }

    // offsets 2..S right inside the segment, where the two ends lie in different runs
    unsigned same = h1;   // bit c: columns c .. c + k joined by offset-1 edges
    unsigned hprev = h1;  // the right word of offset k - 1
#pragma unroll
    for (int k = 2; k <= S; ++k) {
        same &= h1 >> (k - 1);
        const unsigned hk = wd(k, u);
        // via column c + 1 or via column c + k - 1
        unsigned x = hk & ~same & ~((h1 & (hprev >> 1)) | (hprev & (h1 >> (k - 1)))) &
                     (0xffffffffu >> k);
        hprev = hk;
        if (!x) continue;
        const unsigned cuts = rs | (rs >> k);
        do {
            const int c = __ffs(x) - 1;
            op(base + top_bit(rs & upto(c + k)), base + top_bit(rs & upto(c)));
            x = skip_to_next(x, cuts, c);
        } while (x);
    }

    // offsets 1..S into the next segment of the row: bit j of right word k shifted right by
    // 32 - k is the edge from column 32 - k + j to column j of the next segment
    unsigned cross = 0;
#pragma unroll
    for (int k = 1; k <= S; ++k) cross |= wd(k, u) >> (32 - k);
    if (cross) {
        const unsigned rsn = wd.starts(u + 1);
        int la = -1, lb = -1;  // the last pair
#pragma unroll
        for (int k = 1; k <= S; ++k) {
            unsigned x = wd(k, u) >> (32 - k);
            while (x) {
                const int j = __ffs(x) - 1;
                x &= x - 1u;
                const int a = base + top_bit(rs & upto(32 - k + j));
                const int b = base + 32 + top_bit(rsn & upto(j));
                if (a != la || b != lb) {
                    op(b, a);
                    la = a;
                    lb = b;
                }
            }
        }
    }
}

// The diagonal pairs of runs (x, y), y < x, whose upper end lies in row segment u (row r):
// the edges (r, c)-(r+k, c+k) and (r, c)-(r+k, c-k) of its diagonal words.  An edge that a
// vertical offset-k edge and a run of row r or of row r+k already join is dropped — on
// smooth surfaces nearly all of them; of consecutive edges joining the same two runs only
// the first is taken.  Far ends in the next or previous segment of row r+k lie inside the
// strip (the edge pass records no other).
template <int S, class Op>
__device__ __forceinline__ void for_each_diag_pair(const Strip& s, const Words<S>& wd,
                                                   const Words<S>& dd, int u, Op op) {
    const int nsl = s.sh - 5;
    const int NS = 1 << nsl;
    const int r = u >> nsl;
    const unsigned h1 = wd(1, u);
    const unsigned rs = wd.starts(u);
    const int base = u << 5;
#pragma unroll
    for (int k = 1; k <= S; ++k) {
        if (r + k >= s.R) break;
        unsigned dr = dd(k, u), dl = dd(S + k, u);
        if (!(dr | dl)) continue;
        const int ud = u + k * NS;  // the same segment of row r + k
        const unsigned vk = wd(S + k, u);
        const unsigned hd = wd(1, ud);
        // bit c: columns c .. c + k form one run (row r: sa, row r + k: sb)
        unsigned sa = ~0u, sb = ~0u;
#pragma unroll
        for (int j = 0; j < k; ++j) {
            sa &= h1 >> j;
            sb &= hd >> j;
        }
        dr &= ~((vk & sb) | (sa & (vk >> k)));
        dl &= ~((vk & (sb << k)) | ((sa & vk) << k));
        const unsigned rsd = wd.starts(ud);
        int la = -1, lb = -1;
        while (dr) {
            const int c = __ffs(dr) - 1;
            dr &= dr - 1u;
            const int t = c + k;
            const int a = base + top_bit(rs & upto(c));
            const int b = t < 32 ? (ud << 5) + top_bit(rsd & upto(t))
                                 : ((ud + 1) << 5) + top_bit(wd.starts(ud + 1) & upto(t - 32));
            if (a != la || b != lb) {
                op(b, a);
                la = a;
                lb = b;
            }
        }
        la = lb = -1;
        while (dl) {
            const int c = __ffs(dl) - 1;
            dl &= dl - 1u;
            const int t = c - k;
            const int a = base + top_bit(rs & upto(c));
            const int b = t >= 0 ? (ud << 5) + top_bit(rsd & upto(t))
                                 : ((ud - 1) << 5) + top_bit(wd.starts(ud - 1) & upto(t + 32));
            if (a != la || b != lb) {
                op(b, a);
                la = a;
                lb = b;
            }
        }
    }
}

// b. Linking: every run start takes as parent the smallest run that one of its pairs
//    reaches (shared-memory atomicMin, no finds).  Parents are smaller, so this is a
//    forest, and most of the strip's structure is in it before any find runs.
template <int S, bool D>
__device__ void link_runs(const Strip& s, const Carve& sm) {
    const Words<S> wd = words_of<S>(s, sm);
    const Words<S> dd = dwords_of<S>(s, sm);
    const int nsl = s.sh - 5;
    int* par = sm.par;
    for (int u = threadIdx.x; u < wd.n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= s.W) continue;
        auto op = [&](int x, int y) { atomicMin(par + slot(x), y); };
        for_each_pair<S>(s, wd, u, op);
        if constexpr (D) for_each_diag_pair<S>(s, wd, dd, u, op);
    }
}

// c. Every pair united (finds with path halving, atomicMin hooking to the smaller root,
//    retry when a hook loses a race).
template <int S, bool D>
__device__ void unite_runs(const Strip& s, const Carve& sm) {
    const Words<S> wd = words_of<S>(s, sm);
    const Words<S> dd = dwords_of<S>(s, sm);
    const int nsl = s.sh - 5;
    int* par = sm.par;
    for (int u = threadIdx.x; u < wd.n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= s.W) continue;
        auto op = [&](int x, int y) { unite(par, x, y, s); };
        for_each_pair<S>(s, wd, u, op);
        if constexpr (D) for_each_diag_pair<S>(s, wd, dd, u, op);
    }
}

// d. Every run start's entry becomes its root (a read-only walk; the only writer of an
//    entry is the thread of its segment, and it writes the final root).
template <int S>
__device__ void flatten_runs(const Strip& s, const Carve& sm) {
    const Words<S> wd = words_of<S>(s, sm);
    const int nsl = s.sh - 5;
    volatile int* vp = sm.par;
    for (int u = threadIdx.x; u < wd.n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= s.W) continue;
        unsigned x = wd.starts(u);
        while (x) {
            const int node = (u << 5) + __ffs(x) - 1;
            x &= x - 1u;
            int budget = s.limit;
            const int root = find_run_ro(vp, node, budget);
            if (budget <= 0) report_timeout(s.status);
            vp[slot(node)] = root;
        }
    }
}

// e. Every pixel's label: the global index of its run's root.  Lanes take four consecutive
//    pixels of a row (one 16-byte store).
template <int S>
__device__ void write_labels(const Strip& s, const Carve& sm) {
    const Words<S> wd = words_of<S>(s, sm);
    const volatile int* vp = sm.par;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsl = s.sh - 5;
    const bool vec = ((s.C & 3) == 0) && ((s.c0 & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(s.labels) & 15) == 0);
    int last_s = -1, last_root = -1;
    // the global label of the run starting at local pixel st (lanes meet few runs)
    auto root_of = [&](int st) {
        if (st != last_s) {
            last_root = global_of(s, vp[slot(st)]);
            last_s = st;
        }
        return last_root;
    };
    for (int r = warp; r < s.R; r += nwarps) {
        int32_t* out = s.labels + (size_t)r * s.C + s.c0;
        for (int c = lane * 4; c < s.W; c += 128) {
            const int u = (r << nsl) + (c >> 5);
            const int sh = c & 31;  // c is a multiple of 4: the four pixels share a segment
            const unsigned v4 = (wd(0, u) >> sh) & 0xFu;  // no bit is set at or past column W
            int v[4] = {-1, -1, -1, -1};
            if (v4) {
                const unsigned rs = wd.starts(u);
                const unsigned r4 = (rs >> sh) & 0xFu;
                const int base = (u << 5) + sh;
                // a valid pixel that starts no run continues the run of the pixel before it,
                // so one run start is searched for (the first pixel's), the rest are bits
                int root = (v4 & 1u) ? root_of((u << 5) + top_bit(rs & upto(sh))) : -1;
                v[0] = root;
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    if ((r4 >> q) & 1u) root = root_of(base + q);
                    v[q] = ((v4 >> q) & 1u) ? root : -1;
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

// f. Component sizes for the cluster filter (FrameDesc::cnt), after the labels are out:
//    every strip-local root's pixel count, stored at its global index, and its bit in the
//    frame's root bitmask.  The parent entries of the roots become counters, -1 - count (the
//    forest is no longer read): a run start whose entry is negative is a root.  A run is its
//    start and the pixels after it that offset-1 edges join (runs end at their 32-column
//    segment).  One thread per row segment; np = 2S + 1 ballot words per segment.  Inlined
//    (as count_strip): an ABI call in this kernel costs far more than the work (measured).
__device__ __forceinline__ void count_runs(const unsigned* w, int* par, int S, int R, int sh,
                                        int W, int C, int c0, int32_t* cnt, uint32_t* roots) {
    const int np = 2 * S + 1;
    const int n = R << (sh - 5);
    const int nsl = sh - 5;
    auto starts = [&](int u) { return w[u * np] & ~(w[u * np + 1] << 1); };
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= W) continue;  // segment past the strip
        unsigned x = starts(u);
        while (x) {
            const int c = (u << 5) + __ffs(x) - 1;
            x &= x - 1u;
            if (par[slot(c)] == c) par[slot(c)] = -1;
        }
    }
    __syncthreads();
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= W) continue;
        const unsigned ends = ~w[u * np + 1] | 0x80000000u;  // no offset-1 edge to the right
        unsigned x = starts(u);
        int acc_root = -1, acc = 0;  // consecutive runs of one root, summed first
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1u;
            const int c = (u << 5) + b;
            const int len = __ffs(ends >> b);  // pixels b .. the first end at or after b
            const int p = par[slot(c)];
            const int root = p < 0 ? c : p;
            if (root != acc_root) {
                if (acc) atomicSub(par + slot(acc_root), acc);
                acc_root = root;
                acc = 0;
            }
            acc += len;
        }
        if (acc) atomicSub(par + slot(acc_root), acc);
    }
    __syncthreads();
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        if (((u & ((1 << nsl) - 1)) << 5) >= W) continue;
        unsigned x = starts(u);
        while (x) {
            const int c = (u << 5) + __ffs(x) - 1;
            x &= x - 1u;
            const int p = par[slot(c)];
            if (p < 0) {
                const int g = (c >> sh) * C + c0 + (c & ((1 << sh) - 1));
                cnt[g] = -1 - p;
                atomicOr(roots + (g >> 5), 1u << (g & 31));
            }
        }
    }
}

// The strip si of frame f.
__device__ __forceinline__ Strip strip_of(const FrameDesc& f, int si) {
    Strip s{};
    s.range = f.range;
    s.labels = f.labels;
    s.kv = f.kv;
    s.kh = f.kh;
    s.kd = f.kd;
    s.status = f.status;
    s.R = f.rows;
    s.C = f.cols;
    s.S = f.skip;
    s.delta2 = f.delta2;
    s.wrap = f.wrap != 0;
    s.c0 = si * f.strip_w;
    s.W = min(f.strip_w, s.C - s.c0);
    s.sh = f.pitch_log2;
    s.RP = (s.W + s.S + 3) & ~3;
    s.bulk = ((s.C & 3) == 0) && ((s.c0 & 3) == 0) && ((s.W & 3) == 0) &&
             ((reinterpret_cast<uintptr_t>(s.range) & 15) == 0);
    s.limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
    s.gnd = f.rows >= 2 ? f.gnd : nullptr;
    s.gnd_tan = f.gnd_tan;
    s.gnd_height = f.gnd_height;
    s.lattice = f.lattice != 0;
    return s;
}

// Step f for strip si of frame fi of a batch, after its strip pass (the forest and the
// ballot words still in shared memory); nothing when the frame is not counted.
__device__ __forceinline__ void count_strip(const FrameDesc* frames, int fi, int si,
                                         unsigned char* base) {
    if (!frames) return;
    const FrameDesc f = frames[fi];
    if (!f.cnt) return;
    const Strip s = strip_of(f, si);
    const Carve sm = carve(base, s);
    __syncthreads();  // the labels are out
    count_runs(sm.words, sm.par, s.S, s.R, s.sh, s.W, s.C, s.c0, f.cnt, f.roots);
}

// Steps 1 and a to e of a staged strip.
template <int S, bool D>
__device__ void phase1_strip(const Strip& s, const Carve& sm) {
    mask_rows<S, D>(s, sm);
    __syncthreads();  // the staged readings are dead from here on
    if (!D && s.lattice) {
        lattice_words<S>(s, sm);
        __syncthreads();
    }
    init_runs<S>(s, sm);
    __syncthreads();
    link_runs<S, D>(s, sm);
    __syncthreads();
    unite_runs<S, D>(s, sm);
    __syncthreads();
    flatten_runs<S>(s, sm);
    __syncthreads();
    write_labels<S>(s, sm);
}

// The strip pass with the diagonal Map Connections: a function of its own, so that its
// larger register needs stay out of the code of the plain strip pass.
__device__ __noinline__ void phase1_diag(const Strip& s, const Carve& sm) {
    switch (s.S) {
        case 1: phase1_strip<1, true>(s, sm); break;
        case 2: phase1_strip<2, true>(s, sm); break;
        case 3: phase1_strip<3, true>(s, sm); break;
        case 4: phase1_strip<4, true>(s, sm); break;
        case 5: phase1_strip<5, true>(s, sm); break;
        case 6: phase1_strip<6, true>(s, sm); break;
        case 7: phase1_strip<7, true>(s, sm); break;
        default: phase1_strip<8, true>(s, sm); break;
    }
}

__device__ __forceinline__ void phase1(const Strip& s, const Carve& sm) {
    if (s.gnd) phase1_ground(s, sm);
    phase1_clean(s, sm);
    if (s.kd) {  // with the diagonal Map Connections
        phase1_diag(s, sm);
        return;
    }
    switch (s.S) {
        case 1: phase1_strip<1, false>(s, sm); break;
        case 2: phase1_strip<2, false>(s, sm); break;
        case 3: phase1_strip<3, false>(s, sm); break;
        case 4: phase1_strip<4, false>(s, sm); break;
        case 5: phase1_strip<5, false>(s, sm); break;
        case 6: phase1_strip<6, false>(s, sm); break;
        case 7: phase1_strip<7, false>(s, sm); break;
        default: phase1_strip<8, false>(s, sm); break;
    }
}

// P2: the boundary merge of one border (strip b's right edge, to strip b + 1 or across
// the seam to strip 0), by the block that completes the second of its two strips.  The
// crossing edges are split into items (32 rows, source column first + j, offset k) so
// that most warps of the block take one: each lane loads its row's two readings and
// strip-local roots, tests the edge, and of consecutive rows that would unite the same
// pair of roots only the first asks.
__device__ __forceinline__ unsigned long long volatile_load_u64(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

template <int S>
__device__ void border_merge_s(const FrameDesc& f, int* hook, int b, int limit,
                               unsigned long long* pair_set) {
    constexpr int kItems = S * (S + 1) / 2;  // (j, k) with j + k >= S
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int R = f.rows, C = f.cols;
    const int c0 = b * f.strip_w;
    const int W = min(f.strip_w, C - c0);  // >= S (several strips, or C >= S)
    const int first = c0 + W - S;          // first column that has a crossing edge
    const int rblocks = (R + 31) >> 5;
    for (int item = warp; item < rblocks * kItems; item += nwarps) {
        const int rb = item / kItems;
        int q = item - rb * kItems;
        int j = 0;  // source column first + j has the j + 1 offsets S - j .. S
        while (q > j) {
            q -= j + 1;
            ++j;
        }
        const int k = S - j + q;
        int tc = first + j + k;  // target column, past the border (< C + S <= 2C)
        if (tc >= C && f.wrap) tc -= C;
        const int r = (rb << 5) + lane;
        const bool ok = r < R && tc < C;
        const int row = (ok ? r : 0) * C;  // frames hold at most 2^21 pixels
        const float av = ok ? load_range_g(f, r, first + j) : 0.0f;
        const float dv = ok ? load_range_g(f, r, tc) : 0.0f;
        const int ga = ok ? __ldcg(f.labels + row + first + j) : 0;
        const int gb = ok ? __ldcg(f.labels + row + tc) : 0;
        const float K = __ldg(f.kh + (ok ? r : 0) * S + k - 1);
        // the sparse Map Connection: offset S from lattice points, offset 1 from all
        const bool used = !f.lattice || k == 1 ||
                          (k == S && r % S == 0 && (first + j) % S == 0);
        const bool e = used && av > 0.0f && dv > 0.0f && edge_pred(av, dv, K, f.delta2);
        const int pa = __shfl_up_sync(kFull, ga, 1);
        const int pb = __shfl_up_sync(kFull, gb, 1);
        const unsigned em = __ballot_sync(kFull, e);
        // dropped when the row above asks for the same pair
        const bool dup = lane > 0 && ((em >> (lane - 1)) & 1u) && pa == ga && pb == gb;
        if (e && !dup && ga != gb) {
            // other lanes and warps of this block may have united this pair already
            const unsigned long long key =
                ((unsigned long long)(unsigned)ga << 32) | (unsigned)gb;
            const int h = (int)((key * 0x9E3779B97F4A7C15ull) >> 58);  // 64 entries
            if (volatile_load_u64(pair_set + h) != key) {
                int budget = limit;
                union_global(f.labels, ga, gb, budget, hook, f.cols, f.strip_w, f.rows);
                if (budget <= 0) report_timeout(f.status);
                pair_set[h] = key;
            }
        }
    }
}

// The same for a single strip narrower than S (wrapping onto itself): plain loops.
__device__ void border_merge_narrow(const FrameDesc& f, int* hook, int limit) {
    const int R = f.rows, C = f.cols, S = f.skip;
    for (int t = threadIdx.x; t < R * C; t += blockDim.x) {
        const int r = t / C, c = t - r * C;
        const float a = load_range_g(f, r, c);
        if (!(a > 0.0f)) continue;
        for (int k = C - c; k <= S; ++k) {
            if (f.lattice && k != 1 && (k != S || r % S != 0 || c % S != 0)) continue;
            const int tc = (c + k) % C;
            const float d = load_range_g(f, r, tc);
            if (d > 0.0f && edge_pred(a, d, __ldg(f.kh + r * S + k - 1), f.delta2)) {
                int budget = limit;
                union_global(f.labels, __ldcg(f.labels + t), __ldcg(f.labels + (size_t)r * C + tc),
                             budget, hook, f.cols, f.strip_w, f.rows);
                if (budget <= 0) report_timeout(f.status);
            }
        }
    }
}

// The diagonal pairs (§III-B-2) that cross border b, at x = the first column right of it
// (x = cols for the azimuth seam): (r, x-k+j)-(r+k, x+j) down to the right from the last k
// columns of strip b, (r, x+j)-(r+k, x-k+j) down to the left from the first k columns of
// the next strip, j = 0..k-1, columns mod cols.  Every strip is at least S wide, so such a
// pair crosses this border only.
__device__ void border_merge_diag(const FrameDesc& f, int* hook, int b, int limit,
                                  unsigned long long* pair_set) {
    const int R = f.rows, C = f.cols, S = f.skip;
    const int c0 = b * f.strip_w;
    const int x = c0 + min(f.strip_w, C - c0);
    const int per_row = S * (S + 1);  // (k, j, direction): 2k of them per k
    for (int t = threadIdx.x; t < R * per_row; t += blockDim.x) {
        const int r = t / per_row;
        int q = t - r * per_row;
        int k = 1;
        while (q >= 2 * k) {
            q -= 2 * k;
            ++k;
        }
        if (r + k >= R) continue;
        const int j = q >> 1;
        int ca = (q & 1) ? x + j : x - k + j;  // upper end
        int cb = (q & 1) ? x - k + j : x + j;  // lower end
        if (ca >= C) ca -= C;                  // the seam (a border past the last column
        if (cb >= C) cb -= C;                  // exists only with wrap)
        const float av = load_range_g(f, r, ca);
        const float bv = load_range_g(f, r + k, cb);
        if (!(av > 0.0f) || !(bv > 0.0f) ||
            !edge_pred(av, bv, __ldg(f.kd + r * S + k - 1), f.delta2))
            continue;
        const int ga = __ldcg(f.labels + (size_t)r * C + ca);
        const int gb = __ldcg(f.labels + (size_t)(r + k) * C + cb);
        if (ga == gb) continue;
        const unsigned long long key = ((unsigned long long)(unsigned)ga << 32) | (unsigned)gb;
        const int h = (int)((key * 0x9E3779B97F4A7C15ull) >> 58);
        if (volatile_load_u64(pair_set + h) == key) continue;
        int budget = limit;
        union_global(f.labels, ga, gb, budget, hook, f.cols, f.strip_w, f.rows);
        if (budget <= 0) report_timeout(f.status);
        pair_set[h] = key;
    }
}

// The diagonal pairs of a single strip narrower than S that wrap around the seam (the
// edge pass records those whose far column lies inside the strip).
__device__ void border_merge_narrow_diag(const FrameDesc& f, int* hook, int limit) {
    const int R = f.rows, C = f.cols, S = f.skip;
    for (int t = threadIdx.x; t < R * C; t += blockDim.x) {
        const int r = t / C, c = t - r * C;
        const float a = load_range_g(f, r, c);
        if (!(a > 0.0f)) continue;
        for (int k = 1; k <= S && r + k < R; ++k) {
            for (int dir = -1; dir <= 1; dir += 2) {
                const int cc = c + dir * k;
                if (cc >= 0 && cc < C) continue;
                const int tc = ((cc % C) + C) % C;
                const float d = load_range_g(f, r + k, tc);
                if (d > 0.0f && edge_pred(a, d, __ldg(f.kd + r * S + k - 1), f.delta2)) {
                    int budget = limit;
                    union_global(f.labels, __ldcg(f.labels + t),
                                 __ldcg(f.labels + (size_t)(r + k) * C + tc), budget, hook, f.cols, f.strip_w, f.rows);
                    if (budget <= 0) report_timeout(f.status);
                }
            }
        }
    }
}

__device__ void border_merge(const FrameDesc& f, int b, int* hook) {
    const int limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
    // root pairs this block has united during this merge (a cache: a collision only
    // costs a repeated union)
    __shared__ unsigned long long pair_set[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) pair_set[i] = ~0ull;
    __syncthreads();
    const int W = min(f.strip_w, f.cols - b * f.strip_w);
    if (W < f.skip) {
        border_merge_narrow(f, hook, limit);
        if (f.kd) border_merge_narrow_diag(f, hook, limit);
        return;
    }
    if (f.kd) border_merge_diag(f, hook, b, limit, pair_set);
    switch (f.skip) {
        case 1: border_merge_s<1>(f, hook, b, limit, pair_set); break;
        case 2: border_merge_s<2>(f, hook, b, limit, pair_set); break;
        case 3: border_merge_s<3>(f, hook, b, limit, pair_set); break;
        case 4: border_merge_s<4>(f, hook, b, limit, pair_set); break;
        case 5: border_merge_s<5>(f, hook, b, limit, pair_set); break;
        case 6: border_merge_s<6>(f, hook, b, limit, pair_set); break;
        case 7: border_merge_s<7>(f, hook, b, limit, pair_set); break;
        default: border_merge_s<8>(f, hook, b, limit, pair_set); break;
    }
}

// P3: flatten one strip once its frame's forest is final.  A warp takes groups of four
// 128-column row chunks and issues their loads before any find, so that the latency of
// one load round trip covers four chunks.  The roots found are kept in a block-wide cache
// in shared memory (label -> root, one 64-bit entry each, so a reader never sees half of
// an update; a collision only costs a find), so each distinct label of the strip costs
// about one find; in front of it each thread remembers its last lookup.
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// With component sizes (FrameDesc::cnt): each strip-local root of this strip that a border
// merge hooked adds its count to its component's root and leaves the root bitmask, so that
// afterwards the bitmask holds the components' minima and cnt their sizes.  One thread per
// bitmask word of the strip (rows x the words of a row's columns c0 .. c0 + W - 1), all
// loads of the block in flight at once.  Inlined: a real call here costs far more than
// the work (measured).
__device__ __forceinline__ void phase3_counts(int32_t* labels, int32_t* cnt, uint32_t* roots,
                                              int32_t* status, int rows, int cols, int c0,
                                              int W, int limit) {
    const int per_row = ((c0 + W - 1) >> 5) - (c0 >> 5) + 2;  // >= the words a row touches
    const int n = rows * per_row;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = i / per_row;
        const int p_first = r * cols + c0, p_last = p_first + W - 1;
        const int w = (p_first >> 5) + (i - r * per_row);
        if (w > (p_last >> 5)) continue;
        unsigned bits = __ldcg(roots + w);
        if (w == (p_first >> 5)) bits &= ~0u << (p_first & 31);
        if (w == (p_last >> 5)) bits &= (2u << (p_last & 31)) - 1u;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1u;
            const int l = (w << 5) + b;
            int budget = limit;
            const int root = find_global(labels, l, budget, false);
            if (budget <= 0) report_timeout(status);
            if (root != l) {
                atomicAdd(cnt + root, __ldcg(cnt + l));
                atomicAnd(roots + w, ~(1u << b));
            }
        }
    }
}

// r0: the first row that can change (rows above the topmost hooked root keep their labels).
template <bool kCount>
__device__ void phase3_strip(const FrameDesc& f, int si, unsigned long long* cache, int r0) {
    constexpr int G = 4;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int c0 = si * f.strip_w;
    const int W = min(f.strip_w, f.cols - c0);
    const int limit = f.iter_limit > 0 ? f.iter_limit : kDefaultIterLimit;
    const bool vec = ((f.cols & 3) == 0) && ((c0 & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(f.labels) & 15) == 0);
    // cache entries: a power of two, at most 1024, inside this launch's shared memory
    unsigned cn = 1024;
    while (cn > 1 && cn * 8 > dynamic_smem_bytes()) cn >>= 1;
    for (unsigned i = threadIdx.x; i < cn; i += blockDim.x) cache[i] = ~0ull;
    __syncthreads();
    const int nchunk = (W + 127) >> 7;
    const int items = (f.rows - r0) * nchunk;
    int last_l = -1, last_root = -1;
    for (int i0 = warp * G; i0 < items; i0 += nwarps * G) {
        int v[G][4];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int it = i0 + g;
            const int rr = it / nchunk;
            const int c = ((it - rr * nchunk) << 7) + lane * 4;
            const int r = r0 + rr;
            const int32_t* row = f.labels + (size_t)r * f.cols + c0;
            if (it < items && vec && c + 4 <= W) {
                const int4 x = __ldcg(reinterpret_cast<const int4*>(row + c));
                v[g][0] = x.x; v[g][1] = x.y; v[g][2] = x.z; v[g][3] = x.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    v[g][q] = it < items && c + q < W ? __ldcg(row + c + q) : -1;
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int it = i0 + g;
            if (it >= items) break;
            const int rr = it / nchunk;
            const int c = ((it - rr * nchunk) << 7) + lane * 4;
            const int r = r0 + rr;
            bool changed = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int l = v[g][q];
                if (l < 0) continue;
                if (l != last_l) {
                    const unsigned h = ((unsigned)l * 0x9E3779B1u) >> 22 & (cn - 1);
                    const unsigned long long e = ((volatile unsigned long long*)cache)[h];
                    if ((unsigned)(e >> 32) == (unsigned)l) {
                        last_root = (int)(unsigned)e;
                    } else {
                        int budget = limit;
                        last_root = find_global(f.labels, l, budget, false);
                        if (budget <= 0) report_timeout(f.status);
                        cache[h] = ((unsigned long long)(unsigned)l << 32) | (unsigned)last_root;
                    }
                    last_l = l;
                }
                if (last_root != l) {
                    v[g][q] = last_root;
                    changed = true;
                }
            }
            if (changed) {
                int32_t* row = f.labels + (size_t)r * f.cols + c0;
                if (vec && c + 4 <= W) {
                    __stcg(reinterpret_cast<int4*>(row + c),
                           make_int4(v[g][0], v[g][1], v[g][2], v[g][3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c + q < W) __stcg(row + c + q, v[g][q]);
                }
            }
        }
    }
    if (kCount && f.cnt)
        phase3_counts(f.labels, f.cnt, f.roots, f.status, f.rows, f.cols, c0, W, limit);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// kCount: the instance that also counts component sizes (FrameDesc::cnt); the plain
// instance has no trace of it.
template <bool kCount>
__global__ void __launch_bounds__(512, 2) flic_label_kernel(const LabelLaunch L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t tma_bar;
    __shared__ int task_sh;
    __shared__ int flag_sh;
    __shared__ int merge_sh[2];
    __shared__ int p3_row_sh;
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
        // [borders merged, (unused), arrivals at border 0, 1, ...]
        int* done_ctr = L.counters + kCtrFrames + kCtrPerFrame * fi;

        if (kind == kTaskP1) {
            const Strip s = strip_of(f, si);
            const Carve sm = carve(smem_raw, s);
            phase1_stage(s, sm, &tma_bar, parity);
            if (s.bulk) parity ^= 1u;
            phase1(s, sm);
            // (from the descriptor in global memory: nothing of the strip pass stays live)
            if (kCount) count_strip(L.frames, fi, si, smem_raw);
            if (border) {
                // arrive at the (up to two) borders of this strip (both arrivals at once,
                // by two threads); the second arrival at a border merges it.  A merged
                // border adds one to the frame's count with a release reduction, and the
                // frame is ready for P3 when the count reaches its number of borders.
                const int n = f.nstrips;
                const int nb = f.wrap ? n : n - 1;
                __threadfence();
                __syncthreads();
                if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
                    const int side = threadIdx.x >> 5;
                    const int b = side == 0 ? si : si - 1;  // right border, then left border
                    const int bb = b < 0 ? (f.wrap ? n - 1 : -1) : b;
                    int mine = 0;
                    if (bb >= 0 && bb < nb && !(side == 1 && n == 1)) {
                        const int need = n == 1 ? 1 : 2;
                        mine = atomicAdd(done_ctr + 2 + bb, 1) == need - 1 ? bb + 1 : 0;
                    }
                    merge_sh[side] = mine;  // border + 1 to merge, 0 for none
                }
                __syncthreads();
                for (int side = 0; side < 2; ++side) {
                    const int bb = merge_sh[side] - 1;
                    if (bb < 0) continue;  // uniform
                    __threadfence();
                    border_merge(f, bb, done_ctr + kCtrHookRows);
                    __threadfence();
                    __syncthreads();
                    if (threadIdx.x == 0) red_release_add(done_ctr, 1);
                }
            }
        } else {
            if (threadIdx.x == 0) {
                const int nb = f.wrap ? f.nstrips : f.nstrips - 1;
                int it = 0;
                flag_sh = 1;
                while (ld_acquire(done_ctr) < nb) {
                    __nanosleep(128);
                    if (++it > (1 << 24)) {  // ~2 s: give up and leave the strip alone,
                        report_timeout(f.status);  // its labels may not be written yet
                        flag_sh = 0;
                        break;
                    }
                }
                // the topmost row that a merge hooked a root of (the merges are all done)
                p3_row_sh = f.rows - __ldcg(done_ctr + kCtrHookRows + si);
            }
            __syncthreads();
            if (flag_sh)
                phase3_strip<kCount>(f, si, reinterpret_cast<unsigned long long*>(smem_raw),
                                     p3_row_sh);
        }
        __syncthreads();  // shared memory is reused by the next task
    }

    // the last block to leave resets the counters for the next launch on this stream, with
    // all of its threads (one thread alone spent tens of microseconds on a 256-frame batch's
    // 17k counters, after every other block had left)
    if (threadIdx.x == 0) {
        __threadfence();
        flag_sh = atomicAdd(L.counters + kCtrExit, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (flag_sh) {
        const size_t n = counter_ints(nframes);
        for (size_t i = threadIdx.x; i < n; i += blockDim.x) L.counters[i] = 0;
        __threadfence();
    }
}

// flic_edges over 16-byte words: a thread owns one float4 (four adjacent columns) of
// kEdgeRows consecutive rows.  All of its loads come first: the kEdgeRows + S words of its
// column and the one or two words to the right of each of its rows (wrapped modulo the
// row, or past its end without wrap).  A reading that is no measurement, and every word
// beyond the frame, is held as +inf, which fails every test by itself: (a - inf)^2 and
// K (a inf) are +inf or NaN.  So the tests need no validity or bounds checks, and run as
// packed f32x2 pairs of adjacent pixels, each element the scalar sequence of edge_pred.
// The four masks of a row leave as one 8-byte store.  Needs cols % 4 == 0, a 16-byte
// aligned range image, an 8-byte aligned mask and no ground filter; other frames take the
// one-pixel-per-thread kernel below.
constexpr int kEdgeRows = 2;

// (+inf, the one non-measurement that passes x > 0, is already the sentinel)
__device__ __forceinline__ float inf_clean(float x) {
    return x > 0.0f ? x : __int_as_float(0x7f800000);
}

// bit when d <= D2, else 0 (one set and one logic instruction)
__device__ __forceinline__ unsigned bit_le(float d, float D2, unsigned bit) {
    unsigned m;
    asm("set.le.u32.f32 %0, %1, %2;" : "=r"(m) : "f"(d), "f"(D2));
    return m & bit;
}

__device__ __forceinline__ float4 inf_clean4(float4 v) {
    return make_float4(inf_clean(v.x), inf_clean(v.y), inf_clean(v.z), inf_clean(v.w));
}

__device__ __forceinline__ float4 inf4() {
    const float i = __int_as_float(0x7f800000);
    return make_float4(i, i, i, i);
}

// d2 of the pairs (a0, b0) and (a1, b1), both with the constant K.
__device__ __forceinline__ void edge_d2_x2(float a0, float a1, float b0, float b1, float K,
                                           float& d0, float& d1) {
    unsigned long long A, B, KK, t, tt, ab, kab, d2;
    asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b0), "f"(b1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(KK) : "f"(K));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(A), "l"(B));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(tt) : "l"(t));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(ab) : "l"(A), "l"(B));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(kab) : "l"(KK), "l"(ab));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d2) : "l"(tt), "l"(kab));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d2));
}

template <int S>
__global__ void __launch_bounds__(128) flic_edges_vec_kernel(const FrameDesc f,
                                                             uint16_t* __restrict__ mask) {
    const int Q = f.cols >> 2;  // words per row
    const int RT = (f.rows + kEdgeRows - 1) / kEdgeRows;
    const float4* __restrict__ rg = reinterpret_cast<const float4*>(f.range);
    const int total = Q * RT;
    const float D2 = f.delta2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int rt = t / Q;
        const int q = t - rt * Q;
        const int r0 = rt * kEdgeRows;
        const int c0 = q << 2;
        int q1 = q + 1, q2 = q + 2;  // the words holding columns c0+4.. and c0+8..
        const bool in1 = f.wrap || q1 < Q, in2 = f.wrap || q2 < Q;
        while (q1 >= Q) q1 -= Q;
        while (q2 >= Q) q2 -= Q;
        float4 w[kEdgeRows + S], h1[kEdgeRows], h2[kEdgeRows];
#pragma unroll
        for (int i = 0; i < kEdgeRows + S; ++i)
            w[i] = r0 + i < f.rows ? inf_clean4(__ldg(rg + (size_t)(r0 + i) * Q + q)) : inf4();
#pragma unroll
        for (int i = 0; i < kEdgeRows; ++i) {
            const bool row = r0 + i < f.rows;
            h1[i] = row && in1 ? inf_clean4(__ldg(rg + (size_t)(r0 + i) * Q + q1)) : inf4();
            h2[i] = S >= 5 && row && in2 ? inf_clean4(__ldg(rg + (size_t)(r0 + i) * Q + q2))
                                         : inf4();
        }
#pragma unroll
        for (int i = 0; i < kEdgeRows; ++i) {
            const int r = r0 + i;
            if (r >= f.rows) break;
            // row r, columns c0 .. c0 + 11
            const float hv[12] = {w[i].x,  w[i].y,  w[i].z,  w[i].w,  h1[i].x, h1[i].y,
                                  h1[i].z, h1[i].w, h2[i].x, h2[i].y, h2[i].z, h2[i].w};
            unsigned m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
#pragma unroll
            for (int k = 1; k <= S; ++k) {
                const float Kh = __ldg(f.kh + r * S + k - 1);
                const float Kv = r + k < f.rows ? __ldg(f.kv + r * S + k - 1) : 0.0f;
                const unsigned bh = 1u << (k - 1), bv = 1u << (8 + k - 1);
                float d0, d1, d2, d3;
                edge_d2_x2(hv[0], hv[1], hv[k], hv[k + 1], Kh, d0, d1);
                edge_d2_x2(hv[2], hv[3], hv[k + 2], hv[k + 3], Kh, d2, d3);
                m0 |= bit_le(d0, D2, bh);
                m1 |= bit_le(d1, D2, bh);
                m2 |= bit_le(d2, D2, bh);
                m3 |= bit_le(d3, D2, bh);
                const float4& v = w[i + k];
                edge_d2_x2(hv[0], hv[1], v.x, v.y, Kv, d0, d1);
                edge_d2_x2(hv[2], hv[3], v.z, v.w, Kv, d2, d3);
                m0 |= bit_le(d0, D2, bv);
                m1 |= bit_le(d1, D2, bv);
                m2 |= bit_le(d2, D2, bv);
                m3 |= bit_le(d3, D2, bv);
            }
            if (S > 1 && f.lattice) {  // sparse Map Connection: offset 1 everywhere, offset S
                const unsigned far = (1u << (S - 1)) | (1u << (8 + S - 1));  // from lattice
                const bool rok = r % S == 0;                                 // points only
                m0 &= 0x0101u | (rok && (c0 + 0) % S == 0 ? far : 0u);
                m1 &= 0x0101u | (rok && (c0 + 1) % S == 0 ? far : 0u);
                m2 &= 0x0101u | (rok && (c0 + 2) % S == 0 ? far : 0u);
                m3 &= 0x0101u | (rok && (c0 + 3) % S == 0 ? far : 0u);
            }
            uint2 out;
            out.x = m0 | (m1 << 16);
            out.y = m2 | (m3 << 16);
            *reinterpret_cast<uint2*>(mask + (size_t)r * f.cols + c0) = out;
        }
    }
}

// flic_edges: the neighbour test alone, one pixel per thread, straight from global memory.
__global__ void flic_edges_kernel(const FrameDesc f, uint16_t* __restrict__ mask) {
    const int N = f.rows * f.cols;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int r = p / f.cols;
        const int c = p - r * f.cols;
        const float a = load_range_g(f, r, c);
        unsigned m = 0;
        if (a > 0.0f) {
            for (int k = 1; k <= f.skip; ++k) {
                if (f.lattice && k != 1 &&
                    (k != f.skip || r % f.skip != 0 || c % f.skip != 0))
                    continue;  // the sparse Map Connection
                int cc = c + k;
                bool has = true;
                if (cc >= f.cols) {
                    if (f.wrap) cc %= f.cols; else has = false;
                }
                if (has) {
                    const float b = load_range_g(f, r, cc);
                    if (b > 0.0f && edge_pred(a, b, __ldg(f.kh + r * f.skip + k - 1), f.delta2))
                        m |= 1u << (k - 1);
                }
                if (r + k < f.rows) {
                    const float b = load_range_g(f, r + k, c);
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
    cudaError_t e = cudaFuncSetAttribute(flic_label_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flic_label_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
    return e;
}

cudaError_t launch_label(const LabelLaunch& L, int grid, int threads, size_t smem,
                         cudaStream_t stream, bool count) {
    if (count)
        flic_label_kernel<true><<<grid, threads, smem, stream>>>(L);
    else
        flic_label_kernel<false><<<grid, threads, smem, stream>>>(L);
    return cudaGetLastError();
}

cudaError_t label_blocks_per_sm(int threads, size_t smem, int* out) {
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, flic_label_kernel<false>,
                                                                  threads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, flic_label_kernel<true>, threads,
                                                          smem);
    *out = a < b ? a : b;  // one grid size serves both instances
    return e;
}

// One resident wave of 128-thread blocks (grid-stride over the tiles): no second partial
// wave and no ramp between waves.
template <int S>
static cudaError_t launch_edges_vec(const FrameDesc& f, uint16_t* mask, int work,
                                    cudaStream_t stream) {
    static int per_sm[64];  // resident blocks per SM, by device (0: not yet known)
    static int sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) dev = 63;
    if (per_sm[dev] <= 0) {
        int b = 0, n = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, flic_edges_vec_kernel<S>, 128,
                                                               0)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        sms[dev] = n > 0 ? n : 1;
        per_sm[dev] = b > 0 ? b : 1;
    }
    int blocks = (work + 127) / 128;
    blocks = std::max(1, std::min(blocks, per_sm[dev] * sms[dev]));
    flic_edges_vec_kernel<S><<<blocks, 128, 0, stream>>>(f, mask);
    return cudaGetLastError();
}

cudaError_t launch_edges(const FrameDesc& f, uint16_t* mask, cudaStream_t stream) {
    const int N = f.rows * f.cols;
    const int threads = 256;
    const bool vec = f.cols % 4 == 0 && !f.gnd && f.skip >= 1 && f.skip <= 8 &&
                     ((uintptr_t)f.range & 15) == 0 && ((uintptr_t)mask & 7) == 0;
    if (vec) {
        const int work = (f.cols / 4) * ((f.rows + kEdgeRows - 1) / kEdgeRows);
        switch (f.skip) {
            case 1: return launch_edges_vec<1>(f, mask, work, stream);
            case 2: return launch_edges_vec<2>(f, mask, work, stream);
            case 3: return launch_edges_vec<3>(f, mask, work, stream);
            case 4: return launch_edges_vec<4>(f, mask, work, stream);
            case 5: return launch_edges_vec<5>(f, mask, work, stream);
            case 6: return launch_edges_vec<6>(f, mask, work, stream);
            case 7: return launch_edges_vec<7>(f, mask, work, stream);
            default: return launch_edges_vec<8>(f, mask, work, stream);
        }
    }
    int blocks = (N + threads - 1) / threads;
    if (blocks < 1) blocks = 1;
    flic_edges_kernel<<<blocks, threads, 0, stream>>>(f, mask);
    return cudaGetLastError();
}

}  // namespace flic
