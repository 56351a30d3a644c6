// flic_device.cuh — device helpers shared by the FLIC kernels.
#pragma once

#include <cstdint>

#include "flic_internal.h"

namespace flic {

constexpr float kFltMax = 3.402823466e+38f;
constexpr int32_t kStatusTimeout = 4;  // == FLIC_ERR_TIMEOUT

// A range reading is a measurement iff positive and finite (zero = no return, §III-A).
__device__ __forceinline__ bool valid_range(float x) { return x > 0.0f && x <= kFltMax; }

// Read-only load of one range reading; anything that is not a measurement becomes 0.
__device__ __forceinline__ float load_range(const float* p) {
    float x = __ldg(p);
    return valid_range(x) ? x : 0.0f;
}

// Eq. 2 squared in the form (a - b)^2 + K (a b), K = 2 - 2 cos(alpha) (Eq. 3's constant
// without its cancellation), against delta^2.  Every operation is a separately rounded
// fp32 op (explicit _rn intrinsics are never contracted into an FMA), and K multiplies
// the product a*b so that the result is symmetric in (a, b) bit for bit.
__device__ __forceinline__ bool edge_pred(float a, float b, float K, float delta2) {
    float t = __fsub_rn(a, b);
    float tt = __fmul_rn(t, t);
    float ab = __fmul_rn(a, b);
    float kab = __fmul_rn(K, ab);
    float d2 = __fadd_rn(tt, kab);
    return d2 <= delta2;
}

// Two edge tests that share the first reading a — (a, b0, K0) and (a, b1, K1) — as one
// chain of packed fp32x2 operations (sub, mul, mul, mul, add, each element rounded to
// nearest on its own, exactly the scalar sequence of edge_pred): d2 of each pair.
__device__ __forceinline__ void edge_d2_pair(float a, float b0, float b1, float K0, float K1,
                                             float& d0, float& d1) {
    unsigned long long A, B, KK, t, tt, ab, kab, d2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b0), "f"(b1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(KK) : "f"(K0), "f"(K1));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(A), "l"(B));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(tt) : "l"(t));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(ab) : "l"(A), "l"(B));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(kab) : "l"(KK), "l"(ab));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d2) : "l"(tt), "l"(kab));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d2));
}

// ---- ground extraction (§III-A) ---------------------------------------------------------
// d2 spans a horizontal surface with the reading d1 above it when the angle beta of Eq. 1
// (tangent form, the constants of the table row g) lies within the row's bounds:
// num = d2 sin(alpha), den = d1 - d2 cos(alpha), den > 0 and lo*den <= num <= hi*den, every
// operation one fp32 rounding.  Both readings must be measurements (0 for none).
__device__ __forceinline__ bool ground_horizontal(float d1, float d2, const float* g) {
    if (!(d1 > 0.0f) || !(d2 > 0.0f)) return false;
    const float num = __fmul_rn(d2, __ldg(g + 0));
    const float den = __fsub_rn(d1, __fmul_rn(d2, __ldg(g + 1)));
    if (!(den > 0.0f)) return false;
    return num >= __fmul_rn(__ldg(g + 2), den) && num <= __fmul_rn(__ldg(g + 3), den);
}

// A horizontal reading d of a row with table row g is kept (not ground) when it lies above
// the height line z = rho tan(theta) - height (z = d sin(e), rho = d cos(e)).
__device__ __forceinline__ bool ground_above_line(float d, const float* g, float tan_theta,
                                                  float height) {
    if (!(height > 0.0f)) return false;
    const float z = __fmul_rn(d, __ldg(g + 4));
    const float rho = __fmul_rn(d, __ldg(g + 5));
    return z > __fsub_rn(__fmul_rn(rho, tan_theta), height);
}

// A reading of the frame from global memory, 0 where it is no measurement or ground.
// The first row decides as the second (it has no row above).
__device__ __forceinline__ float load_range_g(const FrameDesc& f, int r, int col) {
    const float d = load_range(f.range + (size_t)r * f.cols + col);
    if (!f.gnd || !(d > 0.0f) || f.rows < 2) return d;
    const int rt = r == 0 ? 1 : r;
    const float d1 = load_range(f.range + (size_t)(rt - 1) * f.cols + col);
    const float d2 = rt == r ? d : load_range(f.range + (size_t)rt * f.cols + col);
    if (!ground_horizontal(d1, d2, f.gnd + rt * kGroundFields)) return d;
    if (ground_above_line(d, f.gnd + r * kGroundFields, f.gnd_tan, f.gnd_height)) return d;
    return 0.0f;
}

__device__ __forceinline__ void report_timeout(int32_t* status) {
    if (status) atomicExch(status, kStatusTimeout);
}

// ---- union-find in global memory (the labels buffer holds the cross-strip forest) ------
// Loads bypass L1 (.cg): other blocks write these entries.

__device__ __forceinline__ int find_global(int32_t* lab, int x, int& budget, bool compress) {
    while (true) {
        int p = __ldcg(lab + x);
        if (p == x) return x;
        int gp = __ldcg(lab + p);
        if (gp == p) return p;
        if (compress) __stcg(lab + x, gp);
        x = gp;
        if (--budget <= 0) return x;
    }
}

// hook_rows: per strip of the frame, rows - the topmost row of a root that a union hooked
// (atomicMax, 0: none).  A local component lies at or below its root's row, so the flatten
// of a strip can start at that row: no label above it changes.
__device__ __forceinline__ void union_global(int32_t* lab, int a, int b, int& budget,
                                             int* hook_rows, int cols, int strip_w, int rows) {
    while (budget > 0) {
        a = find_global(lab, a, budget, true);
        b = find_global(lab, b, budget, true);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicMin(lab + b, a);
        if (old == b) {  // root b hooked under a
            atomicMax(hook_rows + (b % cols) / strip_w, rows - b / cols);
            return;
        }
        b = old;
        --budget;
    }
}

// ---- TMA bulk copies into shared memory, completed on an mbarrier ---------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait for the given phase parity; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Order this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (TMA) writes to the same shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One 1-D bulk copy global -> this block's shared memory (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace flic
