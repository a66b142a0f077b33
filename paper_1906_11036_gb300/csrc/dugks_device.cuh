// dugks_device.cuh -- device-side building blocks of the DUGKS step for the
// 2-D NCDE with D2Q9 (arXiv:1906.11036, Section 2).
//
// Notation: P = fbar^+ (Eq. 2.21), Fp = ftilde^+ (Eq. 2.13), phi = sum_i ftilde_i.
// The equilibrium of Eq. 2.3 with B = u b(phi), D = d(phi) I and
// C = u u int_0^phi b'^2 is, per velocity i, a polynomial in phi whose
// coefficients the host computes once (feq[i][m]).
//
// Interface reconstruction (Eqs. 2.19, 2.20, 2.26) at a face between a left
// (or lower) cell L and a right (or upper) cell R, with w = (x_b - x_L)/(x_R - x_L),
// hcd = h c / (x_R - x_L) and tangential weights (tl, tr):
//   fbar_i = [(1-w) + e_n hcd] P_L - e_t hc tl G_L + [w - e_n hcd] P_R - e_t hc tr G_R
// where e_n, e_t are the normal and tangential components of the unit
// velocity direction and G the cell central difference of P along the face.
// Each cell's two halves ("left part" and "right part") are computed by the
// thread that owns the cell, so every face value is a sum of two terms.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dugks {

constexpr int Q = 9;

// D2Q9 direction components in units of c (Eq. 2.5)
__host__ __device__ constexpr int EX(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int EY(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// Per-face reconstruction metrics.
template <typename T>
struct FaceM {
    T w;    // (x_b - x_L) / (x_R - x_L)
    T hcd;  // h c / (x_R - x_L)
    T tl;   // weight of the left cell's tangential slope
    T tr;   // weight of the right cell's tangential slope
};

// Per-cell metrics along one axis.
template <typename T>
struct CellM {
    T ig;  // 1 / (x_{j+1} - x_{j-1}): central-difference factor
    T r;   // dt c / dx_j: flux factor of the cell update
};

template <typename T, int NC>
struct Consts {
    T feq[Q][NC];  // feq_i(phi) = sum_m feq[i][m] phi^m
    T hbp[Q][NC];  // b_bp * feq[i][m]: P = a_bp ft + hbp_i(phi)
    T hf[Q][NC];   // b_f * feq[i][m]: f = a_f fbar + hf_i(phi_b)
    T third;       // 1/3 of Eq. 2.23
    T a_bp, b_bp;  // P  = a_bp ft + b_bp feq   (Eq. 2.21)
    T a_tp, b_tp;  // Fp = a_tp ft + b_tp feq   (Eq. 2.13)
    T a_f, b_f;    // f  = a_f fbar + b_f feq(phi_b) at a face (Eq. 2.22)
    T hc;          // h c, h = dt / 2
    T bcv[4];      // Dirichlet wall values W, E, S, N
};

template <typename T, int NC>
__device__ __forceinline__ T feq_i(const Consts<T, NC>& k, int i, T phi) {
    T s = k.feq[i][NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma(s, phi, k.feq[i][m]);
    return s;
}

// All nine equilibria.  The rest velocity takes feq_0 = phi - sum_{i>0} feq_i
// (zeroth moment of Eq. 2.7), so that rounded weights cannot bias the
// discrete mass in single precision.
template <typename T, int NC>
__device__ __forceinline__ void feq_all(const Consts<T, NC>& k, T phi, T (&out)[Q]) {
    T s = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        out[i] = feq_i(k, i, phi);
        s += out[i];
    }
    out[0] = phi - s;
}

// fbar at a face -> original f for the velocities that cross it
// (interface phi and Eq. 2.22).  NORMAL_X selects x-faces (flux of velocities
// with EX != 0) or y-faces (EY != 0).  Output is packed in velocity order.
template <typename T, int NC, bool NORMAL_X>
__device__ __forceinline__ void face_original(const Consts<T, NC>& k, const T (&fbar)[Q], T (&f6)[6]) {
    T phib = fbar[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) phib += fbar[i];
    int o = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if ((NORMAL_X ? EX(i) : EY(i)) != 0) {
            f6[o] = fma(k.a_f, fbar[i], k.b_f * feq_i(k, i, phib));
            ++o;
        }
    }
}

// index of velocity i among the six that cross an x-face (EX != 0) / y-face (EY != 0)
__host__ __device__ constexpr int XSLOT(int i) {
    return i == 1 ? 0 : i == 3 ? 1 : i == 5 ? 2 : i == 6 ? 3 : i == 7 ? 4 : i == 8 ? 5 : -1;
}
__host__ __device__ constexpr int YSLOT(int i) {
    return i == 2 ? 0 : i == 4 ? 1 : i == 5 ? 2 : i == 6 ? 3 : i == 7 ? 4 : i == 8 ? 5 : -1;
}

// ---------------------------------------------------------------------------
// bounded mbarrier / TMA helpers (sm_90+ PTX; compiled for sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of an mbarrier for at most ~`limit_ns`; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        uint64_t t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > limit_ns) return false;
    }
}
// 3-D tiled TMA load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 4-D tiled TMA load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, uint64_t* bar, int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// a pair of FP32 values on the packed instructions of sm_100+ (__fadd2_rn,
// __fmul2_rn, __ffma2_rn): two opposite velocities of a velocity set
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 f2(float a, float b) { return F2{make_float2(a, b)}; }
__device__ __forceinline__ F2 f2(float a) { return F2{make_float2(a, a)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ F2 shfl_dn2(F2 x) {
    return f2(__shfl_down_sync(0xffffffffu, x.v.x, 1), __shfl_down_sync(0xffffffffu, x.v.y, 1));
}
__device__ __forceinline__ F2 shfl_up2(F2 x) {
    return f2(__shfl_up_sync(0xffffffffu, x.v.x, 1), __shfl_up_sync(0xffffffffu, x.v.y, 1));
}
// (a + s b, a - s b) for the direction sign s of a pair's first velocity
__device__ __forceinline__ F2 sgn2(float a, float b, int s) {
    return s > 0 ? f2(a + b, a - b) : (s < 0 ? f2(a - b, a + b) : f2(a));
}

}  // namespace dugks
