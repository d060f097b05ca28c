// CUDA kernels of libkoma (sm_103a).
//
// K1  bloch_fp32_kernel<S, SPLIT>  spins stepped through the record stream
//                           in FP32, phase in hi/lo FP32, signal partials per
//                           spin range (SPLIT: several CTAs per range divide
//                           its ADC runs).
// K1d bloch_fp64_kernel     the same walk in FP64 (KOMA_FP64).
// K2  reduce_partials<P>    fixed-order sum of the per-CTA partials (FP32 rows by TwoSum).
// K3  bloch_items_kernel<S> grouped phantoms: one warp per work item of one
//                           group, persistent CTAs, per-item partial rows.
// K4  bloch_batches_kernel  serving: batches of many simulations in one
//                           persistent launch (spin ranges of each request).
// K5  bloch_motion_kernel<S, SPLIT>  moving spins, x(t) = x + v t.
// K6  readout_mma_kernel    ADC runs sharing their per-sample rotator, summed
//                           as complex matrix products on the tensor cores
//                           (tcgen05.mma, FP16 hi/lo operands, FP32 in TMEM).
//
// Method: KomaMRI.jl paper, Section "Physical and Mathematical Background"
// (Bloch equation, operator splitting, spinor rotation in the excitation
// regime, e^{i phi} in the precession regime, relaxation) and Section
// "Simulation blocks, Regime Switching, and Sequence-Aware Time Stepping"
// (integral phase over piecewise-linear gradients). The signal at an ADC
// sample is the sum of Mxy over spins (Section "GPU/CPU Parallelization").
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "koma_internal.h"

namespace koma {
namespace {

constexpr int kTile = 64;                 // records per TMA tile (4 KB of Rec32; persistent and motion kernels)
constexpr int kTile1 = 256;               // records per tile of the FP32 Bloch kernel (16 KB: fewer tile barriers)
constexpr int kMaxBlock = 256;
constexpr int kMaxWarps = kMaxBlock / 32;
constexpr int kRed = 128;                 // samples per reduction buffer (FP64 kernel)
constexpr int kRed32 = 512;               // samples per reduction buffer (FP32 kernel, dynamic smem)
constexpr int kV = 8;                     // samples per warp reduce-scatter
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound on any device wait

static_assert(kRed >= kMaxAdcRun && kRed32 >= kMaxAdcRun, "an ADC record must fit in one reduction buffer");
static_assert(kMaxAdcRun % kV == 0, "runs are processed in chunks of kV");

// ---------------------------------------------------------------------------
// sin(pi x), cos(pi x) in FP32.
// Reduction: x = q/2 + r with q = rint(2x) and |r| <= 1/4; r is exact for
// |x| < 2^22. Then sin/cos of t = pi r (|t| <= pi/4) by their Taylor series
// (coefficients 1/n!), truncated where the remainder is below 2e-10, and the
// quadrant q mod 4 selects/negates. Relative error ~1e-7 also for small
// arguments (the hardware sine's absolute error would accumulate over the
// hundreds of small rotations of a soft pulse).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sincospi_f32(float x, float* s, float* c) {
    const float q = rintf(x + x);
    const float r = fmaf(q, -0.5f, x);
    const float t = r * 3.14159265358979323846f;
    const float t2 = t * t;
    float ps = fmaf(t2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);  // 1/9!, -1/7!
    ps = fmaf(ps, t2, 8.33333333333333333e-3f);                              // 1/5!
    ps = fmaf(ps, t2, -1.66666666666666667e-1f);                             // -1/3!
    ps = ps * t2;
    const float sn = fmaf(ps, t, t);
    float pc = fmaf(t2, -2.75573192239858907e-7f, 2.48015873015873016e-5f); // -1/10!, 1/8!
    pc = fmaf(pc, t2, -1.38888888888888889e-3f);                             // -1/6!
    pc = fmaf(pc, t2, 4.16666666666666667e-2f);                              // 1/4!
    pc = fmaf(pc, t2, -0.5f);
    const float cs = fmaf(pc, t2, 1.0f);
    const int iq = static_cast<int>(q);
    const bool swap = iq & 1;
    const float s1 = swap ? cs : sn;
    const float c1 = swap ? sn : cs;
    *s = __int_as_float(__float_as_int(s1) ^ ((iq & 2) << 30));
    *c = __int_as_float(__float_as_int(c1) ^ (((iq + 1) & 2) << 30));
}

// Fractional part (turns) of (ah + al)(bh + bl), to ~1e-7 absolute:
// ah*bh = p + e exactly (FMA), p - rint(p) is exact, and the cross terms are
// small. The integer part of the product is dropped (it is a whole turn).
__device__ __forceinline__ float frac_product(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);
    const float r = p - rintf(p);
    const float c = fmaf(ah, bl, fmaf(al, bh, e));
    return r + c;
}

// e^x - 1 in FP32 with relative accuracy also for small |x| (relaxation over
// one short step, applied many times, must not drift): the Taylor series
// through x^5 for |x| < 1/32 (remainder below 1e-10 relative), else
// exp(x) - 1 where the cancellation costs at most 5 bits.
__device__ __forceinline__ float expm1_f32(float x) {
    if (fabsf(x) < 0.03125f) {
        float p = fmaf(x, 1.f / 120.f, 1.f / 24.f);
        p = fmaf(p, x, 1.f / 6.f);
        p = fmaf(p, x, 0.5f);
        return fmaf(p * x, x, x);
    }
    return expf(x) - 1.f;
}

// ---------------------------------------------------------------------------
// TMA (bulk async copy) + mbarrier helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bulk copy of `bytes` (multiple of 16, 16-byte aligned ends) global -> this
// CTA's shared memory, completing on mbarrier `bar`.
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes,
                                            uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// Order this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Two adjacent mbarriers in shared memory, addressed by index without a
// local-memory array.
struct BarPair {
    uint32_t b0;
    __device__ __forceinline__ uint32_t operator[](int i) const { return b0 + 8u * static_cast<uint32_t>(i); }
};

// Wait for phase `parity` of `bar`, giving up after `limit_ns` (default kWaitNs).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// warp reductions (fixed butterfly order: deterministic)
// ---------------------------------------------------------------------------
// Reduce-scatter of kV = 8 per-lane values: returns, on every lane, the warp
// sum of value index (lane >> 2) & 7.
__device__ __forceinline__ float reduce_scatter8(float (&a)[kV], int lane) {
    const bool b4 = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = b4 ? a[i + 4] : a[i];
        const float send = b4 ? a[i] : a[i + 4];
        a[i] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    const bool b3 = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b3 ? a[i + 2] : a[i];
        const float send = b3 ? a[i] : a[i + 2];
        a[i] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    const bool b2 = lane & 4;
    {
        const float keep = b2 ? a[1] : a[0];
        const float send = b2 ? a[0] : a[1];
        a[0] = keep + __shfl_xor_sync(kFull, send, 4);
    }
    a[0] += __shfl_xor_sync(kFull, a[0], 2);
    a[0] += __shfl_xor_sync(kFull, a[0], 1);
    return a[0];
}

// Compensated FP32 accumulation (Knuth's TwoSum per addition: s + x = t + e
// exactly, with t the rounded sum; the errors e are collected in c). The
// total s + c is exact up to c's own rounding, about n 2^-48 of the sum of
// magnitudes for n terms, instead of the n 2^-24 of a plain FP32 chain.
struct TwoSumAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(s) + static_cast<double>(c); }
    __device__ __forceinline__ float value32() const { return s + c; }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (two spins per 64-bit register pair). fma/mul/add.f32x2
// run at the same FP32 pipe rate as two scalar instructions but take one
// issue slot.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpk(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// -a for both halves: the sign bits flipped by an integer operation (ALU
// pipe, exact), so the FP32 pipe keeps its cycles for arithmetic
__device__ __forceinline__ f32x2 neg2(f32x2 a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// both halves equal
__device__ __forceinline__ f32x2 bcast2(float v) { return pk(v, v); }
// v - rint(v) for both halves (exact)
__device__ __forceinline__ f32x2 frac2(f32x2 v) {
    float a, b;
    unpk(v, a, b);
    return sub2(v, pk(rintf(a), rintf(b)));
}
// frac_product for two spins (a) and one factor (b, both halves equal):
// the same operations as the scalar form, lane by lane
__device__ __forceinline__ f32x2 frac_product2(f32x2 ah, f32x2 al, f32x2 bh, f32x2 bl) {
    const f32x2 p = mul2(ah, bh);
    const f32x2 e = fma2(ah, bh, neg2(p));
    return add2(frac2(p), fma2(ah, bl, fma2(al, bh, e)));
}

// ---------------------------------------------------------------------------
// Per-thread spin set: S spins held in registers for a whole walk of the
// record stream. Slot s is spin base + s * stride when that is < end. Keeps
// M(t_ref) = (mx, my, mz) per spin; parameters are loaded once. A slot past
// the end holds M0 = 0 and zero state and is stepped like the others (its
// values stay 0): no per-slot branch, so the S spins' dependency chains
// interleave.
// ---------------------------------------------------------------------------
template <int S, bool UNI = false>
struct Spins {
    static_assert(S % 2 == 0, "spins are processed in packed pairs");
    static constexpr int NP = S / 2;
    float xh[S], yh[S], zh[S], fh[S], m0[S], r1[S], r2[S];
    float mx[S], my[S], mz[S], em1[S], em2[S], zr[S], zi[S], zr2[S], zi2[S];
    // lo halves of x, y, z, df: in registers for 2 spins per thread (the
    // grouped kernel's usual shape); for 4 (no registers to spare) from a
    // shared-memory copy the kernel made of its slots (`slo`, K1), else from
    // L1 at each exact evaluation
    static constexpr bool kLoRegs = S <= 2;
    float xl[kLoRegs ? S : 1], yl[kLoRegs ? S : 1], zl[kLoRegs ? S : 1], fl[kLoRegs ? S : 1];
    const float* slo = nullptr;  // shared [4][S * stride]: x, y, z, df lo of slot s of thread t at t + s * stride
    int sidx = 0;                // this thread's t
    int64_t base, end;
    int stride;
    float dt_cached;               // em1/em2 belong to this dt
    int rf_mode;                   // rotation path of the current RF run (uniform)
    int rf_terms;                  // series length of the run on the series path (1, 2 or 4)
    bool rf_grad;                  // the run's gradient reaches some spin (else theta_z = pi dt df)
    float key0, key1, key2, key3;  // zr/zi belong to this (dK, dtau)
    float kb0, kb1, kb2, kb3;      // zr2/zi2 belong to this one (the previous run's)
    // every spin of the walk has the same T1 and T2 (a dictionary entry's
    // isochromats): relaxation factors are evaluated once, for slot 0
    static constexpr bool uni = UNI;

    __device__ __forceinline__ int64_t index(int s) const { return base + static_cast<int64_t>(s) * stride; }

    // lo half of a coordinate of slot s: in registers, or in the shared-memory
    // copy every kernel using this path makes at start (slo; zero for slots
    // past the end)
    template <int N>
    __device__ __forceinline__ float lo(const float (&regs)[N], int row, int s) const {
        if constexpr (kLoRegs) {
            return regs[s];
        } else {
            return slo[((row - P32_XL) >> 1) * (S * stride) + sidx + s * stride];
        }
    }

    __device__ __forceinline__ void load(const float* __restrict__ P, int64_t np, int64_t base_, int stride_,
                                         int64_t end_) {
        base = base_;
        stride = stride_;
        end = end_;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = index(s);
            const bool v = j < end;
            xh[s] = v ? P[P32_XH * np + j] : 0.f;
            yh[s] = v ? P[P32_YH * np + j] : 0.f;
            zh[s] = v ? P[P32_ZH * np + j] : 0.f;
            fh[s] = v ? P[P32_FH * np + j] : 0.f;
            m0[s] = v ? P[P32_M0 * np + j] : 0.f;
            r1[s] = v ? P[P32_R1 * np + j] : 0.f;
            r2[s] = v ? P[P32_R2 * np + j] : 0.f;
            if constexpr (kLoRegs) {
                xl[s] = v ? P[P32_XL * np + j] : 0.f;
                yl[s] = v ? P[P32_YL * np + j] : 0.f;
                zl[s] = v ? P[P32_ZL * np + j] : 0.f;
                fl[s] = v ? P[P32_FL * np + j] : 0.f;
            }
            mx[s] = 0.f;
            my[s] = 0.f;
            mz[s] = m0[s];
            em1[s] = 0.f;
            em2[s] = 0.f;
            zr[s] = 1.f;
            zi[s] = 0.f;
            zr2[s] = 1.f;
            zi2[s] = 0.f;
        }
        dt_cached = -1.f;
        rf_mode = 0;
        rf_terms = 4;
        rf_grad = true;
        key0 = __int_as_float(0x7fc00000);  // NaN: no rotator yet
        key1 = key2 = key3 = 0.f;
        kb0 = key0;
        kb1 = kb2 = kb3 = 0.f;
    }

    // Checkpointed state [3][np] (Mx, My, Mz at t_ref) of a walk that was cut.
    __device__ __forceinline__ void load_state(const float* __restrict__ st, int64_t np) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = index(s);
            if (j < end) {
                mx[s] = st[j];
                my[s] = st[np + j];
                mz[s] = st[2 * np + j];
            }
        }
    }
    __device__ __forceinline__ void save_state(float* __restrict__ st, int64_t np) const {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = index(s);
            if (j < end) {
                st[j] = mx[s];
                st[np + j] = my[s];
                st[2 * np + j] = mz[s];
            }
        }
    }

    // A repeated pulse taken by its map: M <- A M + c per spin. The map buffer
    // mp holds, per spin j, the three rows (A_i0, A_i1, A_i2, c_i) as float4
    // at mp4[i * np + j]: three 16-byte loads per spin.
    __device__ __forceinline__ void apply_map(const float* __restrict__ mp, int64_t np) {
        const float4* __restrict__ mp4 = reinterpret_cast<const float4*>(mp);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = index(s);
            if (j < end) {
                const float4 r0 = mp4[j], r1 = mp4[np + j], r2 = mp4[2 * np + j];
                const float x = mx[s], y = my[s], z = mz[s];
                mx[s] = fmaf(r0.x, x, fmaf(r0.y, y, fmaf(r0.z, z, r0.w)));
                my[s] = fmaf(r1.x, x, fmaf(r1.y, y, fmaf(r1.z, z, r1.w)));
                mz[s] = fmaf(r2.x, x, fmaf(r2.y, y, fmaf(r2.z, z, r2.w)));
            }
        }
    }

    // One excitation step for every slot: rotation about the step's constant
    // field, then relaxation over dt. The record holds theta = pi gammabar dt
    // (B1x, B1y, Gbar) and the spin adds pi dt df, so theta is the half-angle
    // vector in radians; the spinor of the step (Eq. Rot_exc, phi = -2|theta|)
    // is the rotation by -2|theta| about theta/|theta|, applied as the
    // quaternion w = cos|theta|, u = -theta sin|theta|/|theta|. General path:
    // |theta| by rsqrt, sin and cos of pi x after exact reduction.
    __device__ __forceinline__ void rf_slots(float gx, float gy, float gz, float bx, float by, float b2, float dt) {
        const float pdt = dt * 3.14159265358979323846f;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float az = fmaf(gx, xh[s], fmaf(gy, yh[s], fmaf(gz, zh[s], fh[s] * pdt)));
            const float t2 = fmaf(az, az, b2);
            const float rs = rsqrtf(t2);
            float ch, sh;
            sincospi_f32(t2 * rs * 0.318309886183790671538f, &sh, &ch);
            const float nsinc = -sh * rs;  // -sin(t)/t
            const float ux = bx * nsinc, uy = by * nsinc, uz = az * nsinc;
            // 2/|q|^2 to first order (keeps |M| from drifting over many steps
            // of one constant field)
            const float nq = fmaf(ch, ch, fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
            const float c2 = fmaf(-2.f, nq, 4.f);
            // v' = v + 2 w (u x v) + 2 u x (u x v)
            const float px = fmaf(uy, mz[s], -uz * my[s]);
            const float py = fmaf(uz, mx[s], -ux * mz[s]);
            const float pz = fmaf(ux, my[s], -uy * mx[s]);
            const float qx = fmaf(uy, pz, -uz * py);
            const float qy = fmaf(uz, px, -ux * pz);
            const float qz = fmaf(ux, py, -uy * px);
            const float nx = fmaf(c2, fmaf(ch, px, qx), mx[s]);
            const float ny = fmaf(c2, fmaf(ch, py, qy), my[s]);
            const float nz = fmaf(c2, fmaf(ch, pz, qz), mz[s]);
            mx[s] = fmaf(em2[s], nx, nx);
            my[s] = fmaf(em2[s], ny, ny);
            mz[s] = fmaf(em1[s], nz - m0[s], nz);
        }
    }

    // Series path (|theta| <= 0.754 for every step and spin): cos t and
    // sin(t)/t as even series in t^2 = theta.theta, so no square root,
    // division or sine is needed; the same rotation and relaxation as
    // rf_slots, on spin pairs in packed f32x2 arithmetic (half the issued
    // instructions). NT = terms after the leading 1, chosen per run from its
    // largest |theta| so the remainder stays below 3e-9 (under half an FP32
    // ulp): NT = 4 (cos to t^10, sinc to t^8) up to 0.754, NT = 2 (t^4, t^4:
    // remainders t^6/720 and t^6/5040) up to 0.1, NT = 1 (t^2, t^2: t^4/24
    // and t^4/120) up to 0.015 — a short excitation pulse's steps.
    template <bool GRAD, int NT>
    __device__ __forceinline__ void rf_pairs_small(float gx, float gy, float gz, float bx, float by, float b2,
                                                   float dt) {
        const float pdt = dt * 3.14159265358979323846f;
        const f32x2 GX = pk(gx, gx), GY = pk(gy, gy), GZ = pk(gz, gz), PDT = pk(pdt, pdt), B2 = pk(b2, b2);
        const f32x2 BX = pk(bx, bx), BY = pk(by, by);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int s0 = 2 * p, s1 = 2 * p + 1;
            const f32x2 F = pk(fh[s0], fh[s1]);
            f32x2 az = mul2(F, PDT);
            if constexpr (GRAD) {
                const f32x2 X = pk(xh[s0], xh[s1]), Y = pk(yh[s0], yh[s1]), Z = pk(zh[s0], zh[s1]);
                az = fma2(GX, X, fma2(GY, Y, fma2(GZ, Z, az)));
            }
            const f32x2 t2 = fma2(az, az, B2);
            f32x2 nsinc, ch;
            if constexpr (NT == 1) {
                nsinc = fma2(t2, pk(1.66666666666666667e-1f, 1.66666666666666667e-1f), pk(-1.0f, -1.0f));
                ch = fma2(t2, pk(-0.5f, -0.5f), pk(1.0f, 1.0f));
            } else if constexpr (NT == 2) {
                const f32x2 q = fma2(t2, pk(-8.33333333333333333e-3f, -8.33333333333333333e-3f),
                                     pk(1.66666666666666667e-1f, 1.66666666666666667e-1f));
                nsinc = fma2(q, t2, pk(-1.0f, -1.0f));
                const f32x2 c = fma2(t2, pk(4.16666666666666667e-2f, 4.16666666666666667e-2f), pk(-0.5f, -0.5f));
                ch = fma2(c, t2, pk(1.0f, 1.0f));
            } else {
                f32x2 q = fma2(t2, pk(-2.75573192239858907e-6f, -2.75573192239858907e-6f),
                               pk(1.98412698412698413e-4f, 1.98412698412698413e-4f));
                q = fma2(q, t2, pk(-8.33333333333333333e-3f, -8.33333333333333333e-3f));
                q = fma2(q, t2, pk(1.66666666666666667e-1f, 1.66666666666666667e-1f));
                nsinc = fma2(q, t2, pk(-1.0f, -1.0f));
                f32x2 c = fma2(t2, pk(-2.75573192239858907e-7f, -2.75573192239858907e-7f),
                               pk(2.48015873015873016e-5f, 2.48015873015873016e-5f));
                c = fma2(c, t2, pk(-1.38888888888888889e-3f, -1.38888888888888889e-3f));
                c = fma2(c, t2, pk(4.16666666666666667e-2f, 4.16666666666666667e-2f));
                c = fma2(c, t2, pk(-0.5f, -0.5f));
                ch = fma2(c, t2, pk(1.0f, 1.0f));
            }
            const f32x2 ux = mul2(BX, nsinc), uy = mul2(BY, nsinc), uz = mul2(az, nsinc);
            const f32x2 nux = neg2(ux), nuy = neg2(uy), nuz = neg2(uz);
            // 2 / |q|^2 to first order; with the two-term series |q|^2 - 1 =
            // -t^4/12 (below 5e-9 here) and the correction multiplies terms
            // of order |theta|, so 2 itself is exact to FP32 rounding
            f32x2 c2 = pk(2.f, 2.f);
            if constexpr (NT > 1) {
                const f32x2 nq = fma2(ch, ch, fma2(ux, ux, fma2(uy, uy, mul2(uz, uz))));
                c2 = fma2(pk(-2.f, -2.f), nq, pk(4.f, 4.f));
            }
            const f32x2 MX = pk(mx[s0], mx[s1]), MY = pk(my[s0], my[s1]), MZ = pk(mz[s0], mz[s1]);
            const f32x2 px = fma2(uy, MZ, mul2(nuz, MY));
            const f32x2 py = fma2(uz, MX, mul2(nux, MZ));
            const f32x2 pz = fma2(ux, MY, mul2(nuy, MX));
            const f32x2 qx = fma2(uy, pz, mul2(nuz, py));
            const f32x2 qy = fma2(uz, px, mul2(nux, pz));
            const f32x2 qz = fma2(ux, py, mul2(nuy, px));
            const f32x2 nx = fma2(c2, fma2(ch, px, qx), MX);
            const f32x2 ny = fma2(c2, fma2(ch, py, qy), MY);
            const f32x2 nz = fma2(c2, fma2(ch, pz, qz), MZ);
            const f32x2 E2 = pk(em2[s0], em2[s1]), E1 = pk(em1[s0], em1[s1]);
            const f32x2 rx = fma2(E2, nx, nx), ry = fma2(E2, ny, ny);
            const f32x2 rz = fma2(E1, sub2(nz, pk(m0[s0], m0[s1])), nz);
            unpk(rx, mx[s0], mx[s1]);
            unpk(ry, my[s0], my[s1]);
            unpk(rz, mz[s0], mz[s1]);
        }
    }

    __device__ __forceinline__ void rf_series(float gx, float gy, float gz, float bx, float by, float b2, float dt) {
        if (rf_grad) {
            if (rf_terms == 1) rf_pairs_small<true, 1>(gx, gy, gz, bx, by, b2, dt);
            else if (rf_terms == 2) rf_pairs_small<true, 2>(gx, gy, gz, bx, by, b2, dt);
            else rf_pairs_small<true, 4>(gx, gy, gz, bx, by, b2, dt);
        } else {
            if (rf_terms == 1) rf_pairs_small<false, 1>(gx, gy, gz, bx, by, b2, dt);
            else if (rf_terms == 2) rf_pairs_small<false, 2>(gx, gy, gz, bx, by, b2, dt);
            else rf_pairs_small<false, 4>(gx, gy, gz, bx, by, b2, dt);
        }
    }

    // Rotation path of an RF run from its header record (see rf()).
    __device__ __forceinline__ void set_mode(const Rec32& H, const float (&ext)[4]) {
        const float mb = H.a[7], mgx = H.a[8], mgy = H.a[9], mgz = H.a[10], mdt = H.a[11];
        const bool same = (mgx == 0.f || ext[0] == 0.f) && (mgy == 0.f || ext[1] == 0.f) &&
                          (mgz == 0.f || ext[2] == 0.f) && ext[3] == 0.f;
        const float bound = mb + mgx * ext[0] + mgy * ext[1] + mgz * ext[2] + mdt * 3.14159265358979323846f * ext[3];
        rf_mode = same ? (mb <= 0.754f ? 3 : 2) : (bound <= 0.754f ? 1 : 0);
        rf_terms = bound <= 0.015f ? 1 : bound <= 0.1f ? 2 : 4;
        rf_grad = (mgx != 0.f && ext[0] != 0.f) || (mgy != 0.f && ext[1] != 0.f) || (mgz != 0.f && ext[2] != 0.f);
    }

    // RF record. The first record of a run of RF records carries the run's
    // maxima; with the phantom's extents `ext` (max |x|, |y|, |z| in m, |df|
    // in Hz) they choose, once per run, between: one rotation for all spins
    // (the field's z part vanishes for every spin; by the series when the
    // run's largest half angle is <= 0.754), the series path (|theta| <= 0.754
    // for every step and spin), or the general path.
    __device__ __forceinline__ void rf(const Rec32& R, const float (&ext)[4]) {
        const float gx = R.a[0], gy = R.a[1], gz = R.a[2];
        const float bx = R.a[3], by = R.a[4], b2 = R.a[5], dt = R.a[6];
        if (R.count > 0) set_mode(R, ext);
        if (dt != dt_cached) {
            // relaxation factors minus one over dt, relatively accurate for
            // short steps (r = log2(e)/T, so -dt/T = -dt r ln 2)
            if (uni) {
                const float a = expm1_f32(-dt * r1[0] * 0.693147180559945309f);
                const float b = expm1_f32(-dt * r2[0] * 0.693147180559945309f);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    em1[s] = a;
                    em2[s] = b;
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    em1[s] = expm1_f32(-dt * r1[s] * 0.693147180559945309f);
                    em2[s] = expm1_f32(-dt * r2[s] * 0.693147180559945309f);
                }
            }
            dt_cached = dt;
        }
        if (rf_mode >= 2)
            rf_uniform(bx, by, b2, rf_mode == 3);
        else if (rf_mode == 1)
            rf_series(gx, gy, gz, bx, by, b2, dt);
        else
            rf_slots(gx, gy, gz, bx, by, b2, dt);
    }

    // RF step whose rotation is the same for every spin (field in the xy
    // plane): quaternion computed once, applied to every slot, then relaxation.
    // SMALL (the run's largest |theta| <= 0.754): cos and sin(t)/t by their
    // even series in t^2 = |theta|^2, as on the per-spin series path.
    __device__ __forceinline__ void rf_uniform(float bx, float by, float b2, bool small) {
        float ch, f;
        if (small) {
            float q = fmaf(b2, -2.75573192239858907e-6f, 1.98412698412698413e-4f);   // -1/9!, 1/7!
            q = fmaf(q, b2, -8.33333333333333333e-3f);                               // -1/5!
            q = fmaf(q, b2, 1.66666666666666667e-1f);                                // 1/3!
            f = fmaf(q, b2, -1.0f);
            float c = fmaf(b2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);  // -1/10!, 1/8!
            c = fmaf(c, b2, -1.38888888888888889e-3f);                               // -1/6!
            c = fmaf(c, b2, 4.16666666666666667e-2f);                                // 1/4!
            c = fmaf(c, b2, -0.5f);
            ch = fmaf(c, b2, 1.0f);
        } else {
            const float rs = rsqrtf(b2);
            float sh;
            sincospi_f32(b2 * rs * 0.318309886183790671538f, &sh, &ch);
            f = -sh * rs;
        }
        const float ux = bx * f, uy = by * f;
        const float nq = fmaf(ch, ch, fmaf(ux, ux, uy * uy));
        const float c2 = fmaf(-2.f, nq, 4.f);
        // u = (ux, uy, 0): p = u x v, q = u x p, on spin pairs in packed f32x2
        const f32x2 UX = pk(ux, ux), UY = pk(uy, uy), NUX = pk(-ux, -ux), NUY = pk(-uy, -uy);
        const f32x2 CH = pk(ch, ch), C2 = pk(c2, c2);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int s0 = 2 * p, s1 = 2 * p + 1;
            const f32x2 MX = pk(mx[s0], mx[s1]), MY = pk(my[s0], my[s1]), MZ = pk(mz[s0], mz[s1]);
            const f32x2 px = mul2(UY, MZ);
            const f32x2 py = mul2(NUX, MZ);
            const f32x2 pz = fma2(UX, MY, mul2(NUY, MX));
            const f32x2 qx = mul2(UY, pz);
            const f32x2 qy = mul2(NUX, pz);
            const f32x2 qz = fma2(UX, py, mul2(NUY, px));
            const f32x2 nx = fma2(C2, fma2(CH, px, qx), MX);
            const f32x2 ny = fma2(C2, fma2(CH, py, qy), MY);
            const f32x2 nz = fma2(C2, fma2(CH, pz, qz), MZ);
            const f32x2 E2 = pk(em2[s0], em2[s1]), E1 = pk(em1[s0], em1[s1]);
            const f32x2 rx = fma2(E2, nx, nx), ry = fma2(E2, ny, ny);
            const f32x2 rz = fma2(E1, sub2(nz, pk(m0[s0], m0[s1])), nz);
            unpk(rx, mx[s0], mx[s1]);
            unpk(ry, my[s0], my[s1]);
            unpk(rz, mz[s0], mz[s1]);
        }
    }

    // Transverse magnetisation at (K, tau) relative to t_ref, per spin:
    // Mxy(t_ref) e^{-tau/T2} e^{-i 2 pi (K.x + df tau)}, the phase's
    // fractional turns from hi/lo products. Terms whose coordinate is zero
    // over the phantom (`used` bits) or whose moment is zero (the record's
    // term bits) are skipped.
    // With `prec` the reference moves to (K, tau) (Mz recovers with T1).
    __device__ __forceinline__ void exact(const Rec32& R, bool prec, const float* __restrict__ P, int64_t np,
                                          int used, float (&er)[S], float (&ei)[S]) {
        const float kxh = R.a[0], kxl = R.a[1], kyh = R.a[2], kyl = R.a[3];
        const float kzh = R.a[4], kzl = R.a[5], th = R.a[6], tl = R.a[7];
        const int terms = (R.count >> kTermShift) & used;
        const bool ux = terms & 1, uy = terms & 2, uz = terms & 4, uf = terms & 8;
        // the decays of every slot, or once when all spins share T1 and T2
        float e2u = 0.f, e1u = 0.f;
        if (uni) {
            e2u = exp2f(-th * r2[0]);
            if (prec) e1u = exp2f(-th * r1[0]);
        }
        if (ux || uy || uz || uf) {
            // the phase's terms, each a uniform branch around all slots
            float F[S];
#pragma unroll
            for (int s = 0; s < S; ++s) F[s] = 0.f;
            if (ux) {
#pragma unroll
                for (int s = 0; s < S; ++s) F[s] += frac_product(xh[s], lo(xl, P32_XL, s), kxh, kxl);
            }
            if (uy) {
#pragma unroll
                for (int s = 0; s < S; ++s) F[s] += frac_product(yh[s], lo(yl, P32_YL, s), kyh, kyl);
            }
            if (uz) {
#pragma unroll
                for (int s = 0; s < S; ++s) F[s] += frac_product(zh[s], lo(zl, P32_ZL, s), kzh, kzl);
            }
            if (uf) {
#pragma unroll
                for (int s = 0; s < S; ++s) F[s] += frac_product(fh[s], lo(fl, P32_FL, s), th, tl);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) {
                // one-shot phase: reduce to [-1/2, 1/2] turn and use the
                // hardware sine (absolute error ~4e-7, not accumulated: every
                // run and every materialisation starts from an exact evaluation)
                const float r = F[s] - rintf(F[s]);
                float sn, cs;
                __sincosf(-6.28318530717958647692f * r, &sn, &cs);
                const float e2 = uni ? e2u : exp2f(-th * r2[s]);
                er[s] = e2 * fmaf(mx[s], cs, -my[s] * sn);
                ei[s] = e2 * fmaf(mx[s], sn, my[s] * cs);
            }
        } else {  // no phase since t_ref (a sample or a pause with no moment and no off-resonance)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float e2 = uni ? e2u : exp2f(-th * r2[s]);
                er[s] = e2 * mx[s];
                ei[s] = e2 * my[s];
            }
        }
        if (prec) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float e1 = uni ? e1u : exp2f(-th * r1[s]);
                mx[s] = er[s];
                my[s] = ei[s];
                mz[s] = fmaf(mz[s] - m0[s], e1, m0[s]);
            }
        }
    }

    // ADC record of L samples starting from (er, ei): sums over the warp's
    // spins of every sample, handed to sink(i, re, im) on one lane per sample
    // (i = sample index within the run). Samples after the first come from
    // the per-sample rotator z = e^{-dtau/T2} e^{-i 2 pi (dK.x + df dtau)}
    // (exact in exact arithmetic for uniformly spaced samples), spins in
    // packed pairs; warp sums by a fixed butterfly (deterministic).
    template <class Sink>
    __device__ __forceinline__ void adc(const Rec32& R, int L, float (&er)[S], float (&ei)[S], int lane,
                                        Sink&& sink) {
        if (L == 1) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                sr += er[s];
                si += ei[s];
            }
            sr = warp_sum(sr);
            si = warp_sum(si);
            if (lane == 0) sink(0, sr, si);
            return;
        }
        const float dkx = R.a[8], dky = R.a[9], dkz = R.a[10], dtau = R.a[11];
        // two cached rotators: alternating runs (an EPI's two readout
        // directions) reuse both
        if (!(dkx == key0 && dky == key1 && dkz == key2 && dtau == key3)) {
            if (dkx == kb0 && dky == kb1 && dkz == kb2 && dtau == kb3) {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const float a = zr[s], b = zi[s];
                    zr[s] = zr2[s];
                    zi[s] = zi2[s];
                    zr2[s] = a;
                    zi2[s] = b;
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    zr2[s] = zr[s];
                    zi2[s] = zi[s];
                    const float th1 = -fmaf(dkx, xh[s], fmaf(dky, yh[s], fmaf(dkz, zh[s], fh[s] * dtau)));
                    float sn, cs;
                    sincospi_f32(2.f * th1, &sn, &cs);
                    const float mag = exp2f(-dtau * r2[s]);
                    zr[s] = mag * cs;
                    zi[s] = mag * sn;
                }
            }
            kb0 = key0;
            kb1 = key1;
            kb2 = key2;
            kb3 = key3;
            key0 = dkx;
            key1 = dky;
            key2 = dkz;
            key3 = dtau;
        }
        f32x2 pr[NP], pi_[NP], qr[NP], qi[NP], qn[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            pr[p] = pk(er[2 * p], er[2 * p + 1]);
            pi_[p] = pk(ei[2 * p], ei[2 * p + 1]);
            qr[p] = pk(zr[2 * p], zr[2 * p + 1]);
            qi[p] = pk(zi[2 * p], zi[2 * p + 1]);
            qn[p] = pk(-zi[2 * p], -zi[2 * p + 1]);
        }
        for (int c = 0; c < L; c += kV) {
            float ar[kV], ai[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                f32x2 sr2 = pr[0], si2 = pi_[0];
#pragma unroll
                for (int p = 1; p < NP; ++p) {
                    sr2 = add2(sr2, pr[p]);
                    si2 = add2(si2, pi_[p]);
                }
                float r0, r1, i0, i1;
                unpk(sr2, r0, r1);
                unpk(si2, i0, i1);
                ar[v] = r0 + r1;
                ai[v] = i0 + i1;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const f32x2 nr2 = fma2(pr[p], qr[p], mul2(pi_[p], qn[p]));
                    pi_[p] = fma2(pr[p], qi[p], mul2(pi_[p], qr[p]));
                    pr[p] = nr2;
                }
            }
            const float sr = reduce_scatter8(ar, lane);
            const float si = reduce_scatter8(ai, lane);
            const int vl = (lane >> 2) & 7;
            if ((lane & 3) == 0 && c + vl < L) sink(c + vl, sr, si);
        }
    }
};

// Tile pipeline of the record stream: 64-record tiles brought into shared
// memory by TMA bulk copies, double buffered; tile g of the CTA's lifetime
// sits in buffer g & 1 and completes phase (g >> 1) & 1 of its mbarrier.
template <int T, class Bars>
__device__ __forceinline__ void issue_tile(Rec32 (*s_rec)[T], const Bars& bar, const Rec32* grec,
                                           int64_t n_rec, int64_t t, uint64_t g) {
    const int64_t nr = min(static_cast<int64_t>(T), n_rec - t * T);
    tma_load_1d(smem_u32(&s_rec[g & 1][0]), grec + t * T, static_cast<uint32_t>(nr * sizeof(Rec32)),
                bar[g & 1]);
}

// ---------------------------------------------------------------------------
// K1: FP32 split-phase Bloch kernel.
//
// Every CTA owns a contiguous spin range; thread `tid` holds spins
// begin + s * blockDim + tid for s < S in registers for the whole sequence.
// All threads walk the same record stream (tiles in shared memory) and read
// each record as a broadcast.
//   RF   rotate by the step's constant field and relax (one step).
//   PREC replace M(t_ref) by M(t) at the given (K, tau).
//   ADC  `count` samples (Spins::adc).
// Warp sample sums are staged per warp in shared memory and summed over
// warps in a fixed order (compensated) into one FP32 partial per (CTA,
// sample). Within a warp the sum over its 32 S spins is a fixed binary tree
// (the S spins of a thread, then the butterfly) of depth log2(32 S): its
// error is at most that depth times 2^-24 of the sum of magnitudes, however
// many spins the launch has; every longer chain of additions (over warps,
// CTAs) is compensated.
// ---------------------------------------------------------------------------
template <int S, bool SPLIT>
__global__ void __launch_bounds__(kMaxBlock, 2) bloch_fp32_kernel(const __grid_constant__ BlochArgs A) {
    __shared__ __align__(128) Rec32 s_rec[2][kTile1];
    __shared__ __align__(8) uint64_t s_bar[2];
    // per-warp sample sums, two buffers: [buf][warp][kRed32] (dynamic)
    extern __shared__ __align__(16) float2 s_red_dyn[];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nthr = blockDim.x;
    const int nwarps = nthr >> 5;
    const int cta = blockIdx.x;
    // ADC-run split: CTAs cta = spin_cta * split + part share one spin range;
    // part p handles the ADC records whose index is p mod split
    const int split = SPLIT ? A.split : 1;
    const int part = SPLIT ? cta % split : 0, scta = SPLIT ? cta / split : cta;

    int64_t c_begin, c_end;
    if (A.cta_begin) {
        c_begin = A.cta_begin[scta];
        c_end = A.cta_begin[scta + 1];
    } else {
        c_begin = static_cast<int64_t>(scta) * A.spins_per_cta;
        c_end = min(A.n, c_begin + A.spins_per_cta);
    }
    const int64_t np = A.n_pad;
    Spins<S> sp;
    sp.load(A.p32, np, c_begin + tid, nthr, c_end);
    // the lo halves of the CTA's spins, read at every exact evaluation
    __shared__ float s_lo[Spins<S>::kLoRegs ? 1 : 4 * S * kMaxBlock];
    if constexpr (!Spins<S>::kLoRegs) {
        for (int i = tid; i < S * nthr; i += nthr) {
            const int64_t j = c_begin + i;
            const bool v = j < c_end;
            s_lo[0 * S * nthr + i] = v ? A.p32[P32_XL * np + j] : 0.f;
            s_lo[1 * S * nthr + i] = v ? A.p32[P32_YL * np + j] : 0.f;
            s_lo[2 * S * nthr + i] = v ? A.p32[P32_ZL * np + j] : 0.f;
            s_lo[3 * S * nthr + i] = v ? A.p32[P32_FL * np + j] : 0.f;
        }
        sp.slo = s_lo;
        sp.sidx = tid;
    }

    int red_buf = 0;
    int64_t red_base = 0, red_end = 0;  // samples [red_base, red_end) staged
    int mma_snap_row = 0;               // snapshot rows stored so far
    // one partial row per spin range; with a split each part writes the
    // samples of its own runs (s_own marks them in the staged window)
    __shared__ unsigned char s_own[SPLIT ? 2 : 1][SPLIT ? kRed32 : 1];
    float2* __restrict__ partial = static_cast<float2*>(A.partial) + static_cast<int64_t>(scta) * A.n_adc;
    auto red_slot = [&](int buf, int w, int i) -> float2& { return s_red_dyn[(buf * nwarps + w) * kRed32 + i]; };
    auto flush = [&]() {
        __syncthreads();
        const int cnt = static_cast<int>(red_end - red_base);
        for (int i = tid; i < cnt; i += nthr) {
            if (SPLIT && !s_own[red_buf][i]) continue;
            // the warps' sums added by TwoSum: the CTA's total is rounded once
            TwoSumAcc sr, si;
            for (int w = 0; w < nwarps; ++w) {
                const float2 v = red_slot(red_buf, w, i);
                sr.add(v.x);
                si.add(v.y);
            }
            partial[red_base + i] = make_float2(sr.value32(), si.value32());
        }
        red_buf ^= 1;
        red_base = red_end;
    };

    const uint32_t bar[2] = {smem_u32(&s_bar[0]), smem_u32(&s_bar[1])};
    const Rec32* __restrict__ grec = static_cast<const Rec32*>(A.rec);
    const int64_t n_tiles = (A.n_rec + kTile1 - 1) / kTile1;
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int64_t t = 0; t < 2 && t < n_tiles; ++t) issue_tile(s_rec, bar, grec, A.n_rec, t, t);
    }

    for (int64_t t = 0; t < n_tiles; ++t) {
        const int b = static_cast<int>(t & 1);
        const bool ok = mbar_wait_bounded(bar[b], static_cast<uint32_t>((t >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            // a tile never arrived: report, wait (bounded) for the copies in
            // flight into this CTA's shared memory, and leave
            if (tid == 0) {
                atomicOr(A.status, kStatusTimeout);
                mbar_wait_bounded(bar[b], static_cast<uint32_t>((t >> 1) & 1));
                if (t + 1 < n_tiles) mbar_wait_bounded(bar[b ^ 1], static_cast<uint32_t>(((t + 1) >> 1) & 1));
            }
            return;
        }
        const int nr = static_cast<int>(min(static_cast<int64_t>(kTile1), A.n_rec - t * kTile1));
        for (int r = 0; r < nr; ++r) {
            const Rec32& R = s_rec[b][r];
            const int type = R.type;
            if (type == REC_RF) {
                sp.rf(R, A.ext);
            } else if (type == REC_MAP) {
                // a repeated pulse as a whole (compacted stream)
                if (R.k0 >= 0 && R.k0 < A.n_rf_maps)
                    sp.apply_map(A.rf_maps + R.k0 * kRfMapFloats * np, np);
                else if (tid == 0)
                    atomicOr(A.status, kStatusBadMap);
            } else if (type == REC_PREC) {
                float er[S], ei[S];
                sp.exact(R, true, A.p32, np, A.used, er, ei);
            } else if (type == REC_ADC) {
                const bool own = !SPLIT || (t * kTile1 + r) % split == part;
                if (A.mma_snap != nullptr && (R.count & kMmaFlag)) {
                    // a run of the matrix-form readout: not sampled here and not
                    // staged (its samples of this CTA's row are never read); the
                    // first of its block stores the block's Mxy(t_ref)
                    if (R.count & kMmaSnapFlag) {
                        if (mma_snap_row >= A.n_mma_snaps) {
                            if (tid == 0) atomicOr(A.status, kStatusBadSnap);
                        } else if (own) {
                            float2* __restrict__ row = A.mma_snap + static_cast<int64_t>(mma_snap_row) * np;
#pragma unroll
                            for (int s = 0; s < S; ++s) {
                                const int64_t j = sp.index(s);
                                if (j < sp.end)
                                    row[j] = make_float2(sp.mx[s] * A.mma_escale, sp.my[s] * A.mma_escale);
                            }
                        }
                        ++mma_snap_row;
                    }
                    continue;
                }
                const int L = min(max(R.count & kCountMask, 1), kMaxAdcRun);
                const int64_t k0 = R.k0;
                if (k0 < red_base || k0 + L > A.n_adc) {  // inside the row, not before the staged window
                    if (tid == 0) atomicOr(A.status, kStatusBadAdc);
                    continue;
                }
                if (k0 + L > red_base + kRed32) {
                    flush();
                    // samples skipped since (matrix-form runs) are not this row's
                    red_base = k0;
                }
                const int off = static_cast<int>(k0 - red_base);
                if (SPLIT && warp == 0)
                    for (int i = lane; i < L; i += 32) s_own[red_buf][off + i] = own;
                if (own) {
                    float er[S], ei[S];
                    sp.exact(R, false, A.p32, np, A.used, er, ei);
                    sp.adc(R, L, er, ei, lane, [&](int i, float sr, float si) {
                        red_slot(red_buf, warp, off + i) = make_float2(sr, si);
                    });
                }
                red_end = k0 + L;
            }
        }
        __syncthreads();  // everyone is done with tile buffer b
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async_smem();
            issue_tile(s_rec, bar, grec, A.n_rec, t + 2, t + 2);
        }
    }
    if (red_end > red_base) flush();
}

// ---------------------------------------------------------------------------
// K7: maps of repeated RF pulses (pre-pass of K1).
//
// For pulse p (a run of RF records that recurs unchanged) and spin j the
// whole run is the affine map M -> A M + c, the composition of its steps
// (rotation about the step's field by the quaternion of the Bloch kernel's
// RF step, then relaxation). The kernel steps the three columns of A (from
// the unit vectors, relaxation without the recovery term) and c (from
// M = 0, with it) through the pulse's records, two spins per thread in
// packed FP32 pairs, and writes maps[p] as float4 rows (row i of A, c_i) per spin. The
// rotation path per run follows the Bloch kernel: cos and sin(t)/t by their
// even series when the run's largest half angle allows it (bound from the
// run header's maxima and the phantom's extents), else rsqrt and sin/cos of
// pi x after exact reduction; the quaternion is renormalised to first order
// on every path.
//
// Precision: A is applied at every occurrence of the pulse, so its rounding
// error repeats identically shot after shot and adds up through the T1
// memory of the magnetisation, where the rounding of stepped pulses differs
// from shot to shot. The columns of A are therefore carried as unevaluated
// FP32 pairs hi + lo: each step's increment (rotation and relaxation, small
// next to the column for the small per-step angles of a soft pulse) is
// computed in FP32 and added to hi by TwoSum, its rounding error going to
// lo, and lo is rotated with the same quaternion. A's error is then that of
// the increments themselves, far below one FP32 rounding of the column per
// step. c (of the order of the recovery over one pulse) needs no pair.
// ---------------------------------------------------------------------------
constexpr int kMapChunk = 128;   // records staged in shared memory at a time
constexpr int kMapBlock = 256;

struct MapPair {
    f32x2 X, Y, Z, F, M0, R1, R2;  // spin parameters of the pair
    f32x2 E1, E2;                   // relaxation factors minus one over dt_cached
    float dt_cached;
    f32x2 v[kRfMapFloats];          // columns of A (x, y, z parts), then c
    f32x2 lo[9];                    // low parts of the columns of A

    // One RF step of the pair: quaternion (w = ch, u), then the four
    // vectors rotated and relaxed. NT: series terms (0: general path).
    template <bool GRAD, int NT>
    __device__ __forceinline__ void step(const Rec32& R) {
        const float dt = R.a[6];
        if (dt != dt_cached) {
            float r1a, r1b, r2a, r2b;
            unpk(R1, r1a, r1b);
            unpk(R2, r2a, r2b);
            const float k = -dt * 0.693147180559945309f;
            E1 = pk(expm1_f32(k * r1a), expm1_f32(k * r1b));
            E2 = pk(expm1_f32(k * r2a), expm1_f32(k * r2b));
            dt_cached = dt;
        }
        const float pdt = dt * 3.14159265358979323846f;
        f32x2 az = mul2(F, pk(pdt, pdt));
        if constexpr (GRAD)
            az = fma2(pk(R.a[0], R.a[0]), X, fma2(pk(R.a[1], R.a[1]), Y, fma2(pk(R.a[2], R.a[2]), Z, az)));
        const float b2 = R.a[5];
        const f32x2 t2 = fma2(az, az, pk(b2, b2));
        f32x2 nsinc, ch;
        if constexpr (NT == 0) {
            float ta, tb, sa, ca, sb, cb;
            unpk(t2, ta, tb);
            const float ra = rsqrtf(ta), rb = rsqrtf(tb);
            sincospi_f32(ta * ra * 0.318309886183790671538f, &sa, &ca);
            sincospi_f32(tb * rb * 0.318309886183790671538f, &sb, &cb);
            nsinc = pk(-sa * ra, -sb * rb);
            ch = pk(ca, cb);
        } else if constexpr (NT == 1) {
            nsinc = fma2(t2, pk(1.66666666666666667e-1f, 1.66666666666666667e-1f), pk(-1.0f, -1.0f));
            ch = fma2(t2, pk(-0.5f, -0.5f), pk(1.0f, 1.0f));
        } else if constexpr (NT == 2) {
            const f32x2 q = fma2(t2, pk(-8.33333333333333333e-3f, -8.33333333333333333e-3f),
                                 pk(1.66666666666666667e-1f, 1.66666666666666667e-1f));
            nsinc = fma2(q, t2, pk(-1.0f, -1.0f));
            const f32x2 c = fma2(t2, pk(4.16666666666666667e-2f, 4.16666666666666667e-2f), pk(-0.5f, -0.5f));
            ch = fma2(c, t2, pk(1.0f, 1.0f));
        } else {
            f32x2 q = fma2(t2, pk(-2.75573192239858907e-6f, -2.75573192239858907e-6f),
                           pk(1.98412698412698413e-4f, 1.98412698412698413e-4f));
            q = fma2(q, t2, pk(-8.33333333333333333e-3f, -8.33333333333333333e-3f));
            q = fma2(q, t2, pk(1.66666666666666667e-1f, 1.66666666666666667e-1f));
            nsinc = fma2(q, t2, pk(-1.0f, -1.0f));
            f32x2 c = fma2(t2, pk(-2.75573192239858907e-7f, -2.75573192239858907e-7f),
                           pk(2.48015873015873016e-5f, 2.48015873015873016e-5f));
            c = fma2(c, t2, pk(-1.38888888888888889e-3f, -1.38888888888888889e-3f));
            c = fma2(c, t2, pk(4.16666666666666667e-2f, 4.16666666666666667e-2f));
            c = fma2(c, t2, pk(-0.5f, -0.5f));
            ch = fma2(c, t2, pk(1.0f, 1.0f));
        }
        const f32x2 ux = mul2(pk(R.a[3], R.a[3]), nsinc), uy = mul2(pk(R.a[4], R.a[4]), nsinc);
        const f32x2 uz = mul2(az, nsinc);
        // 2 / |q|^2 to first order (|u|^2 = t^2 sinc^2): the map is applied
        // many times, so its rotation part is kept orthogonal to FP32
        // rounding on every path
        const f32x2 nq = fma2(ch, ch, mul2(mul2(nsinc, nsinc), t2));
        const f32x2 c2 = fma2(pk(-2.f, -2.f), nq, pk(4.f, 4.f));
        // the step's rotation minus the identity, R - I = c2 (w [u]x + u u^T -
        // |u|^2 I) (the quaternion update v + c2 (w u x v + u x (u x v)) as a
        // matrix), built once and applied to the seven vectors
        const f32x2 cx = mul2(c2, ux), cy = mul2(c2, uy), cz = mul2(c2, uz);
        const f32x2 wx = mul2(cx, ch), wy = mul2(cy, ch), wz = mul2(cz, ch);
        const f32x2 sxy = mul2(cx, uy), sxz = mul2(cx, uz), syz = mul2(cy, uz);
        const f32x2 qx = mul2(cx, ux), qy = mul2(cy, uy), qz = mul2(cz, uz);
        const f32x2 Mxx = neg2(add2(qy, qz)), Myy = neg2(add2(qx, qz)), Mzz = neg2(add2(qx, qy));
        const f32x2 Mxy = sub2(sxy, wz), Myx = add2(sxy, wz);
        const f32x2 Mxz = add2(sxz, wy), Mzx = sub2(sxz, wy);
        const f32x2 Myz = sub2(syz, wx), Mzy = add2(syz, wx);
        // with the relaxation folded in: the whole step is m -> m + N m (+ the
        // recovery on z for c), N = (I + E)(I + M) - I = M + E (I + M) with
        // E = diag(E2, E2, E1) (the relaxation factors minus one)
        const f32x2 Nxx = fma2(E2, Mxx, add2(Mxx, E2)), Nyy = fma2(E2, Myy, add2(Myy, E2));
        const f32x2 Nzz = fma2(E1, Mzz, add2(Mzz, E1));
        const f32x2 Nxy = fma2(E2, Mxy, Mxy), Nxz = fma2(E2, Mxz, Mxz);
        const f32x2 Nyx = fma2(E2, Myx, Myx), Nyz = fma2(E2, Myz, Myz);
        const f32x2 Nzx = fma2(E1, Mzx, Mzx), Nzy = fma2(E1, Mzy, Mzy);
        // hi + lo += d for one component (Fast2Sum: exact while |hi| >= |d|,
        // the case of the small per-step increments compensation is for;
        // otherwise within one rounding of d itself)
        auto acc = [](f32x2& h, f32x2& l, f32x2 d) {
            const f32x2 t = add2(h, d);
            l = add2(l, sub2(d, sub2(t, h)));
            h = t;
        };
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            // columns of A (no recovery term): the increment N m is added to
            // hi; lo follows the same step exactly (m + N m, no rounding to
            // recover there: lo is far below hi's resolution)
            const f32x2 X = v[3 * q], Y = v[3 * q + 1], Z = v[3 * q + 2];
            const f32x2 dx = fma2(Nxx, X, fma2(Nxy, Y, mul2(Nxz, Z)));
            const f32x2 dy = fma2(Nyx, X, fma2(Nyy, Y, mul2(Nyz, Z)));
            const f32x2 dz = fma2(Nzx, X, fma2(Nzy, Y, mul2(Nzz, Z)));
            const f32x2 LX = lo[3 * q], LY = lo[3 * q + 1], LZ = lo[3 * q + 2];
            lo[3 * q] = fma2(Nxx, LX, fma2(Nxy, LY, fma2(Nxz, LZ, LX)));
            lo[3 * q + 1] = fma2(Nyx, LX, fma2(Nyy, LY, fma2(Nyz, LZ, LY)));
            lo[3 * q + 2] = fma2(Nzx, LX, fma2(Nzy, LY, fma2(Nzz, LZ, LZ)));
            acc(v[3 * q], lo[3 * q], dx);
            acc(v[3 * q + 1], lo[3 * q + 1], dy);
            acc(v[3 * q + 2], lo[3 * q + 2], dz);
        }
        {
            // c: the same step plus the recovery M0 (1 - e^{-dt/T1}) = -E1 M0 on z
            const f32x2 X = v[9], Y = v[10], Z = v[11];
            v[9] = fma2(Nxx, X, fma2(Nxy, Y, fma2(Nxz, Z, X)));
            v[10] = fma2(Nyx, X, fma2(Nyy, Y, fma2(Nyz, Z, Y)));
            v[11] = fma2(Nzx, X, fma2(Nzy, Y, fma2(Nzz, Z, fma2(neg2(E1), M0, Z))));
        }
    }
};

template <bool GRAD, int NT>
__device__ __forceinline__ void map_chunk(MapPair& m, const Rec32* s_rec, int n) {
    for (int r = 0; r < n; ++r) m.template step<GRAD, NT>(s_rec[r]);
}

__global__ void __launch_bounds__(kMapBlock) rf_map_kernel(const __grid_constant__ RfMapArgs A) {
    __shared__ __align__(16) Rec32 s_rec[kMapChunk];
    const int tid = threadIdx.x;
    const RfMapPulse P = A.pulses[blockIdx.y];
    const int64_t np = A.n_pad;
    const int64_t j0 = static_cast<int64_t>(blockIdx.x) * (2 * kMapBlock) + tid, j1 = j0 + kMapBlock;
    const bool v0 = j0 < A.n, v1 = j1 < A.n;
    const float* __restrict__ Pp = A.p32;
    auto ld = [&](int row, int64_t j, bool v) { return v ? Pp[row * np + j] : 0.f; };
    MapPair m;
    m.X = pk(ld(P32_XH, j0, v0), ld(P32_XH, j1, v1));
    m.Y = pk(ld(P32_YH, j0, v0), ld(P32_YH, j1, v1));
    m.Z = pk(ld(P32_ZH, j0, v0), ld(P32_ZH, j1, v1));
    m.F = pk(ld(P32_FH, j0, v0), ld(P32_FH, j1, v1));
    m.M0 = pk(ld(P32_M0, j0, v0), ld(P32_M0, j1, v1));
    m.R1 = pk(ld(P32_R1, j0, v0), ld(P32_R1, j1, v1));
    m.R2 = pk(ld(P32_R2, j0, v0), ld(P32_R2, j1, v1));
    m.dt_cached = -1.f;
    m.E1 = m.E2 = pk(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kRfMapFloats; ++k) m.v[k] = pk(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) m.lo[k] = pk(0.f, 0.f);
    m.v[0] = m.v[4] = m.v[8] = pk(1.f, 1.f);  // identity columns

    // rotation path of the run, from its header (as the Bloch kernel's set_mode)
    const Rec32 H = A.rec[P.rec_begin];
    const float mb = H.a[7], mgx = H.a[8], mgy = H.a[9], mgz = H.a[10], mdt = H.a[11];
    const float bound = mb + mgx * A.ext[0] + mgy * A.ext[1] + mgz * A.ext[2] +
                        mdt * 3.14159265358979323846f * A.ext[3];
    const bool grad = (mgx != 0.f && A.ext[0] != 0.f) || (mgy != 0.f && A.ext[1] != 0.f) ||
                      (mgz != 0.f && A.ext[2] != 0.f);
    const int nt = bound > 0.754f ? 0 : bound <= 0.015f ? 1 : bound <= 0.1f ? 2 : 4;

    const uint4* __restrict__ src = reinterpret_cast<const uint4*>(A.rec + P.rec_begin);
    uint4* dst = reinterpret_cast<uint4*>(s_rec);
    for (int c0 = 0; c0 < P.len; c0 += kMapChunk) {
        const int n = min(kMapChunk, P.len - c0);
        __syncthreads();  // the previous chunk's reads are done
        for (int i = tid; i < n * 4; i += kMapBlock) dst[i] = src[static_cast<int64_t>(c0) * 4 + i];
        __syncthreads();
        if (grad) {
            switch (nt) {
                case 0: map_chunk<true, 0>(m, s_rec, n); break;
                case 1: map_chunk<true, 1>(m, s_rec, n); break;
                case 2: map_chunk<true, 2>(m, s_rec, n); break;
                default: map_chunk<true, 4>(m, s_rec, n); break;
            }
        } else {
            switch (nt) {
                case 0: map_chunk<false, 0>(m, s_rec, n); break;
                case 1: map_chunk<false, 1>(m, s_rec, n); break;
                case 2: map_chunk<false, 2>(m, s_rec, n); break;
                default: map_chunk<false, 4>(m, s_rec, n); break;
            }
        }
    }
    // row i of A (A[i][k] = i-th part of column k) and c_i as one float4 per
    // spin: out4[i * np + j]
    float4* __restrict__ out4 = reinterpret_cast<float4*>(A.maps + static_cast<int64_t>(blockIdx.y) * kRfMapFloats * np);
    float a0[kRfMapFloats], a1[kRfMapFloats];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) unpk(add2(m.v[3 * k + i], m.lo[3 * k + i]), a0[3 * i + k], a1[3 * i + k]);
#pragma unroll
    for (int i = 0; i < 3; ++i) unpk(m.v[9 + i], a0[9 + i], a1[9 + i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (v0) out4[i * np + j0] = make_float4(a0[3 * i], a0[3 * i + 1], a0[3 * i + 2], a0[9 + i]);
        if (v1) out4[i * np + j1] = make_float4(a1[3 * i], a1[3 * i + 1], a1[3 * i + 2], a1[9 + i]);
    }
}

// One batch of a persistent kernel: every warp of the CTA steps its own spin
// range [wb, we) of one phantom through records [rb, re) of one record
// stream (TMA tiles shared by the CTA, restarted per batch; `g0` counts the
// tiles the CTA consumed before) and writes its per-sample sums to `row` (if
// not null). A walk that does not start at record 0 resumes from the
// checkpoint `state` (inside an RF run, the run's header `rf_hdr` sets the
// RF path exactly as an unsplit walk had it);
// one that stops before the end saves it there. Returns false if a tile never
// arrived (status set, copies waited for).
template <int S, int T = kTile, bool UNI = false>
__device__ __forceinline__ bool walk_batch(Rec32 (*s_rec)[T], const BarPair bar, uint64_t& g0,
                                           const float* __restrict__ p32, int64_t np, const Rec32* grec,
                                           int64_t n_rec, int64_t rb, int64_t re, float* state, int64_t rf_hdr,
                                           const float (&ext)[4], int used, int64_t wb, int64_t we,
                                           float2* __restrict__ row, int64_t n_adc, int* status,
                                           float* warp_lo, const float* rf_maps = nullptr, int n_maps = 0) {
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const Rec32* base = grec + rb;
    const int64_t n_walk = re - rb;
    const int64_t n_tiles = (n_walk + T - 1) / T;
    Spins<S, UNI> sp;
    sp.load(p32, np, wb + lane, 32, we);
    if constexpr (!Spins<S, UNI>::kLoRegs) {
        // the lo halves of the warp's spins, read at every exact evaluation
        __syncwarp();  // the previous batch's reads of warp_lo are done
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = wb + lane + 32 * s;
            const bool v = j < we;
            warp_lo[0 * S * 32 + lane + 32 * s] = v ? p32[P32_XL * np + j] : 0.f;
            warp_lo[1 * S * 32 + lane + 32 * s] = v ? p32[P32_YL * np + j] : 0.f;
            warp_lo[2 * S * 32 + lane + 32 * s] = v ? p32[P32_ZL * np + j] : 0.f;
            warp_lo[3 * S * 32 + lane + 32 * s] = v ? p32[P32_FL * np + j] : 0.f;
        }
        __syncwarp();
        sp.slo = warp_lo;
        sp.sidx = lane;
    }
    if (state && rb > 0) {
        sp.load_state(state, np);
        if (rf_hdr >= 0) sp.set_mode(grec[rf_hdr], ext);
    }
    if (tid == 0) {
        for (int64_t t = 0; t < 2 && t < n_tiles; ++t) issue_tile(s_rec, bar, base, n_walk, t, g0 + t);
    }
    for (int64_t t = 0; t < n_tiles; ++t) {
        const uint64_t g = g0 + t;
        const int b = static_cast<int>(g & 1);
        const bool ok = mbar_wait_bounded(bar[b], static_cast<uint32_t>((g >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(status, kStatusTimeout);
                mbar_wait_bounded(bar[b], static_cast<uint32_t>((g >> 1) & 1));
                if (t + 1 < n_tiles) mbar_wait_bounded(bar[b ^ 1], static_cast<uint32_t>(((g + 1) >> 1) & 1));
            }
            return false;
        }
        const int nr = static_cast<int>(min(static_cast<int64_t>(T), n_walk - t * T));
        for (int r = 0; r < nr; ++r) {
            const Rec32& R = s_rec[b][r];
            const int type = R.type;
            if (type == REC_RF) {
                sp.rf(R, ext);
            } else if (type == REC_MAP) {
                // a repeated pulse as a whole (compacted stream)
                if (R.k0 >= 0 && R.k0 < n_maps)
                    sp.apply_map(rf_maps + R.k0 * kRfMapFloats * np, np);
                else if (tid == 0)
                    atomicOr(status, kStatusBadMap);
            } else if (type == REC_PREC) {
                float er[S], ei[S];
                sp.exact(R, true, p32, np, used, er, ei);
            } else if (type == REC_ADC) {
                const int L = min(max(R.count & kCountMask, 1), kMaxAdcRun);
                const int64_t k0 = R.k0;
                if (k0 < 0 || k0 + L > n_adc) {
                    if (tid == 0) atomicOr(status, kStatusBadAdc);
                    continue;
                }
                float er[S], ei[S];
                sp.exact(R, false, p32, np, used, er, ei);
                sp.adc(R, L, er, ei, lane, [&](int i, float sr, float si) {
                    if (row) row[k0 + i] = make_float2(sr, si);
                });
            }
        }
        __syncthreads();  // everyone is done with tile buffer b
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async_smem();
            issue_tile(s_rec, bar, base, n_walk, t + 2, g + 2);
        }
    }
    if (state && re < n_rec) sp.save_state(state, np);
    g0 += static_cast<uint64_t>(n_tiles);
    return true;
}

// ---------------------------------------------------------------------------
// K3: grouped ("dictionary") kernel, persistent.
//
// Work item = up to 32 * S spins of one group. One warp steps one item
// through the whole record stream and writes the item's signal as its own
// FP32 partial row; K2 then sums each group's item rows in a fixed order.
// CTAs take batches of (warps per CTA) items from a global counter; the item
// order is longest first, so a batch's items have similar sizes and the last
// batches are the shortest. All warps of a CTA walk the record stream
// together (shared TMA tiles).
// ---------------------------------------------------------------------------
template <int S, int T, bool UNI>
__global__ void __launch_bounds__(kMaxBlock, 2) bloch_items_kernel(const __grid_constant__ ItemArgs A) {
    __shared__ __align__(128) Rec32 s_rec[2][T];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ float s_lo_w[Spins<S>::kLoRegs ? 1 : kMaxWarps * 4 * S * 32];  // per-warp lo halves
    __shared__ int64_t s_batch;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const BarPair bar{smem_u32(&s_bar[0])};
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        fence_mbar_init();
    }
    uint64_t g0 = 0;
    for (;;) {
        if (tid == 0) s_batch = atomicAdd(A.counter, 1);
        __syncthreads();
        const int64_t batch = s_batch;
        __syncthreads();
        if (batch * nwarps >= A.n_items) break;
        const int64_t oi = batch * nwarps + warp;
        int64_t ib = 0, ie = 0;
        float2* row = nullptr;
        if (oi < A.n_items) {
            const int64_t item = A.order[oi];
            ib = A.item_begin[item];
            ie = A.item_begin[item + 1];
            row = static_cast<float2*>(A.partial) + item * A.n_adc;
        }
        if (!walk_batch<S, T, UNI>(s_rec, bar, g0, A.p32, A.n_pad, static_cast<const Rec32*>(A.rec), A.n_rec, 0,
                                   A.n_rec, nullptr, -1, A.ext, A.used, ib, ie, row, A.n_adc, A.status,
                                   s_lo_w + warp * (4 * S * 32)))
            return;
    }
}

// ---------------------------------------------------------------------------
// K3z: grouped kernel for dictionaries of isochromats along z.
//
// When the spins of a phantom differ only in z (x = y = 0 and no off-resonance
// anywhere), every group has a single T1 and T2, the sequence's RF steps carry
// no z gradient (so every RF step rotates all spins alike) and every ADC record
// holds one sample, a spin needs no more state than M, its z and M0, and the
// record work that is the same for all spins is shared by 8 spins per thread.
// The kernel walks its own copy of the record stream, prepared on the host:
// an RF record carries the step's rotation matrix (a[0..8], the renormalised
// quaternion rotation of the uniform RF path of K1/K3, evaluated once per
// record instead of by every thread) and its dt (a[9]), a PREC/ADC record
// -2 pi Kz in a[8].
// A thread steps one unit of up to 8 consecutive spins of one group; units
// are packed across groups (a warp's lanes may hold several groups, a group
// may span warps), so slots are filled to within 8 spins per group. A
// sample's sum is a segmented butterfly over the warp's lanes, one partial
// row per (warp, group) segment; K2 sums a group's rows in order.
// The spins' phase rotators are kept while the phase records' Kz repeats (a
// FISP train's identical unbalanced lobes), as the relaxation factors are
// kept per RF dt.
// SMALLPH (the host checked |z Kz| <= 1 turn for every spin and record): the
// phase angle is z (-2 pi Kz) in one FP32 product, relative error a few ulp of
// an angle of at most 2 pi; otherwise the hi/lo fractional product of K1/K3.
// Relaxation and the sine are applied as in K1/K3.
// ---------------------------------------------------------------------------
constexpr int kZS = 8;             // spins per thread
constexpr int kZNP = kZS / 2;      // packed pairs

constexpr int kZSmallBlock = 128;  // the SMALLPH instances: 5 CTAs of 128 threads per SM (<= 96 registers)

template <int T, bool SMALLPH>
__global__ void __launch_bounds__(SMALLPH ? kZSmallBlock : kMaxBlock, SMALLPH ? 5 : 2) bloch_items_z_kernel(const __grid_constant__ ItemArgs A) {
    __shared__ __align__(128) Rec32 s_rec[2][T];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int64_t s_batch;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const BarPair bar{smem_u32(&s_bar[0])};
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        fence_mbar_init();
    }
    const int64_t np = A.n_pad;
    const float* __restrict__ P = A.p32;
    const Rec32* grec = static_cast<const Rec32*>(A.rec);
    const int64_t n_tiles = (A.n_rec + T - 1) / T;
    uint64_t g0 = 0;
    for (;;) {
        // a batch: blockDim.x consecutive units, one per thread
        if (tid == 0) s_batch = atomicAdd(A.counter, 1);
        __syncthreads();
        const int64_t batch = s_batch;
        __syncthreads();
        if (batch * blockDim.x >= A.n_units) break;
        // this lane's unit: spins [sb, sb + cnt) of one group, item `item`
        const int64_t u = batch * blockDim.x + tid;
        int64_t sb = 0;
        int cnt = 0, item = -1;
        if (u < A.n_units) {
            sb = A.unit_begin[u];
            cnt = static_cast<int>(A.unit_begin[u + 1] - sb);
            item = A.unit_item[u];
        }
        // the warp's segments (runs of lanes with one item): bit k of `same`
        // when lane + 2^k has this lane's item; the segment's first lane
        // writes the item's partial row
        unsigned same = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int o = __shfl_down_sync(kFull, item, 1 << k);
            if (lane + (1 << k) < 32 && item >= 0 && o == item) same |= 1u << k;
        }
        const int prev = __shfl_up_sync(kFull, item, 1);
        float2* row = nullptr;
        if (item >= 0 && (lane == 0 || prev != item))
            row = static_cast<float2*>(A.partial) + static_cast<int64_t>(item) * A.n_adc;
        // the unit's 8 slots: spin sb + s for s < cnt, zero state past it
        f32x2 MX[kZNP], MY[kZNP], MZ[kZNP], ZH[kZNP], ZL[kZNP], M0[kZNP];
#pragma unroll
        for (int p = 0; p < kZNP; ++p) {
            const int64_t j0 = sb + 2 * p, j1 = j0 + 1;
            const bool v0 = 2 * p < cnt, v1 = 2 * p + 1 < cnt;
            ZH[p] = pk(v0 ? P[P32_ZH * np + j0] : 0.f, v1 ? P[P32_ZH * np + j1] : 0.f);
            if (!SMALLPH) ZL[p] = pk(v0 ? P[P32_ZL * np + j0] : 0.f, v1 ? P[P32_ZL * np + j1] : 0.f);
            M0[p] = pk(v0 ? P[P32_M0 * np + j0] : 0.f, v1 ? P[P32_M0 * np + j1] : 0.f);
            MX[p] = pk(0.f, 0.f);
            MY[p] = pk(0.f, 0.f);
            MZ[p] = M0[p];
        }
        // the unit's group shares T1 and T2
        const float r1 = cnt > 0 ? P[P32_R1 * np + sb] : 0.f, r2 = cnt > 0 ? P[P32_R2 * np + sb] : 0.f;
        // relaxation factors minus one (Q1, Q2) for the last RF dt; the spins' phase
        // rotators for the last phase record's Kz (hi, lo): a train of
        // identical lobes (FISP) evaluates them once
        f32x2 Q1 = 0, Q2 = 0;
        float dt_cached = -1.f, kh_cached = 0.f, kl_cached = 0.f;
        bool rot_ok = false;
        f32x2 CS[kZNP], SN[kZNP];
        if (tid == 0) {
            for (int64_t t = 0; t < 2 && t < n_tiles; ++t) issue_tile(s_rec, bar, grec, A.n_rec, t, g0 + t);
        }
        for (int64_t t = 0; t < n_tiles; ++t) {
            const uint64_t g = g0 + t;
            const int b = static_cast<int>(g & 1);
            const bool ok = mbar_wait_bounded(bar[b], static_cast<uint32_t>((g >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(A.status, kStatusTimeout);
                    mbar_wait_bounded(bar[b], static_cast<uint32_t>((g >> 1) & 1));
                    if (t + 1 < n_tiles) mbar_wait_bounded(bar[b ^ 1], static_cast<uint32_t>(((g + 1) >> 1) & 1));
                }
                return;
            }
            const int nr = static_cast<int>(min(static_cast<int64_t>(T), A.n_rec - t * T));
            for (int r = 0; r < nr; ++r) {
                const Rec32& R = s_rec[b][r];
                const int type = R.type;
                if (type == REC_RF) {
                    const float dt = R.a[9];
                    if (dt != dt_cached) {
                        Q1 = bcast2(expm1_f32(-dt * r1 * 0.693147180559945309f));
                        Q2 = bcast2(expm1_f32(-dt * r2 * 0.693147180559945309f));
                        dt_cached = dt;
                    }
                    const f32x2 A00 = bcast2(R.a[0]), A01 = bcast2(R.a[1]), A02 = bcast2(R.a[2]);
                    const f32x2 A10 = bcast2(R.a[3]), A11 = bcast2(R.a[4]), A12 = bcast2(R.a[5]);
                    const f32x2 A20 = bcast2(R.a[6]), A21 = bcast2(R.a[7]), A22 = bcast2(R.a[8]);
#pragma unroll
                    for (int p = 0; p < kZNP; ++p) {
                        const f32x2 nx = fma2(A02, MZ[p], fma2(A01, MY[p], mul2(A00, MX[p])));
                        const f32x2 ny = fma2(A12, MZ[p], fma2(A11, MY[p], mul2(A10, MX[p])));
                        const f32x2 nz = fma2(A22, MZ[p], fma2(A21, MY[p], mul2(A20, MX[p])));
                        MX[p] = fma2(Q2, nx, nx);
                        MY[p] = fma2(Q2, ny, ny);
                        MZ[p] = fma2(Q1, sub2(nz, M0[p]), nz);
                    }
                } else if (type == REC_PREC || type == REC_ADC) {
                    const bool prec = type == REC_PREC;
                    const float th = R.a[6];
                    const bool uz = ((R.count >> kTermShift) & A.used) & 4;
                    const f32x2 E2 = bcast2(exp2f(-th * r2));
                    f32x2 ER[kZNP], EI[kZNP];
                    if (uz) {
                        const float kh = R.a[4], kl = R.a[5];
                        if (!rot_ok || kh != kh_cached || kl != kl_cached) {
                            const f32x2 KH = bcast2(kh), KL = bcast2(kl), W = bcast2(R.a[8]);
#pragma unroll
                            for (int p = 0; p < kZNP; ++p) {
                                float s0, c0, s1, c1;
                                if (SMALLPH) {
                                    float t0, t1;
                                    unpk(mul2(ZH[p], W), t0, t1);
                                    __sincosf(t0, &s0, &c0);
                                    __sincosf(t1, &s1, &c1);
                                } else {
                                    const f32x2 F = frac_product2(ZH[p], ZL[p], KH, KL);
                                    float f0, f1;
                                    unpk(F, f0, f1);
                                    __sincosf(-6.28318530717958647692f * (f0 - rintf(f0)), &s0, &c0);
                                    __sincosf(-6.28318530717958647692f * (f1 - rintf(f1)), &s1, &c1);
                                }
                                SN[p] = pk(s0, s1);
                                CS[p] = pk(c0, c1);
                            }
                            kh_cached = kh;
                            kl_cached = kl;
                            rot_ok = true;
                        }
#pragma unroll
                        for (int p = 0; p < kZNP; ++p) {
                            ER[p] = mul2(E2, fma2(MX[p], CS[p], neg2(mul2(MY[p], SN[p]))));
                            EI[p] = mul2(E2, fma2(MX[p], SN[p], mul2(MY[p], CS[p])));
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < kZNP; ++p) {
                            ER[p] = mul2(E2, MX[p]);
                            EI[p] = mul2(E2, MY[p]);
                        }
                    }
                    if (prec) {
                        const f32x2 E1 = bcast2(exp2f(-th * r1));
#pragma unroll
                        for (int p = 0; p < kZNP; ++p) {
                            MX[p] = ER[p];
                            MY[p] = EI[p];
                            MZ[p] = fma2(sub2(MZ[p], M0[p]), E1, M0[p]);
                        }
                    } else {
                        const int64_t k0 = R.k0;
                        if (k0 < 0 || k0 >= A.n_adc || (R.count & kCountMask) > 1) {
                            if (tid == 0) atomicOr(A.status, kStatusBadAdc);
                            continue;
                        }
                        f32x2 sr2 = ER[0], si2 = EI[0];
#pragma unroll
                        for (int p = 1; p < kZNP; ++p) {
                            sr2 = add2(sr2, ER[p]);
                            si2 = add2(si2, EI[p]);
                        }
                        float a0, a1, c0, c1;
                        unpk(sr2, a0, a1);
                        unpk(si2, c0, c1);
                        float sr = a0 + a1, si = c0 + c1;
                        // segmented sum over the warp's lanes (each lane adds
                        // the partial 2^k lanes up while that lane is in its
                        // segment): the segment's first lane ends with the
                        // segment's total, in a fixed order
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const float ur = __shfl_down_sync(kFull, sr, 1 << k);
                            const float ui = __shfl_down_sync(kFull, si, 1 << k);
                            if ((same >> k) & 1) {
                                sr += ur;
                                si += ui;
                            }
                        }
                        if (row) row[k0] = make_float2(sr, si);
                    }
                }
            }
            __syncthreads();  // everyone is done with tile buffer b
            if (tid == 0 && t + 2 < n_tiles) {
                fence_proxy_async_smem();
                issue_tile(s_rec, bar, grec, A.n_rec, t + 2, g + 2);
            }
        }
        g0 += static_cast<uint64_t>(n_tiles);
    }
}

// ---------------------------------------------------------------------------
// K4: serving kernel, persistent. Batches come from a table that mixes the
// simulations admitted by the server: batch = a contiguous spin range of one
// request's phantom, walked through a chunk of that request's records
// (checkpointed between chunks); warp w of the batch takes the w-th 32 * S
// spins and writes row w of the batch's rows.
// Many simulations thereby share one launch; each request's decomposition
// into batches does not depend on what else is in the launch.
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(kMaxBlock, 2) bloch_batches_kernel(const __grid_constant__ BatchArgs A) {
    __shared__ __align__(128) Rec32 s_rec[2][kTile];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ float s_lo_w[Spins<S>::kLoRegs ? 1 : kMaxWarps * 4 * S * 32];  // per-warp lo halves
    __shared__ int64_t s_batch;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const BarPair bar{smem_u32(&s_bar[0])};
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        fence_mbar_init();
    }
    uint64_t g0 = 0;
    const int64_t n_batches = *A.n_batches_dev;
    for (;;) {
        if (tid == 0) s_batch = atomicAdd(A.counter, 1);
        __syncthreads();
        const int64_t batch = s_batch;
        __syncthreads();
        if (batch >= n_batches) break;
        const BatchDesc& D = A.desc[batch];
        const int64_t per_warp = 32LL * S;
        const int64_t wb = min(D.spin_begin + warp * per_warp, D.spin_end);
        const int64_t we = min(wb + per_warp, D.spin_end);
        float2* row = D.rows + static_cast<int64_t>(warp) * D.n_adc;
        const float ext[4] = {D.ext[0], D.ext[1], D.ext[2], D.ext[3]};
        if (!walk_batch<S>(s_rec, bar, g0, D.p32, D.n_pad, D.rec, D.n_rec, D.rec_begin, D.rec_end, D.state,
                           D.rf_hdr, ext, D.used, wb, we, row, D.n_adc, A.status, s_lo_w + warp * (4 * S * 32),
                           D.rf_maps, D.n_rf_maps))
            return;
    }
}

// ---------------------------------------------------------------------------
// K5: FP32 kernel for moving phantoms, x(t) = x + v t.
//
// The walk of K1 over RecM records. What motion changes:
//   RF    the step's field uses the spin's position at the step midpoint
//         t_mid: az = theta_G.(x + v t_mid) + pi dt df.
//   phase from t_ref to t: 2 pi (K.x + K1.v + df tau), every product in
//         hi/lo (K1 grows with absolute time, so K1.v can be many turns).
//   ADC   the phase increment from sample l to l + 1 is phi1 + l phi2 with
//         phi1 = dK.x + dK1_0.v + df dtau and phi2 = dtau dK.v, so the
//         per-sample rotator itself turns by e^{-i 2 pi phi2} every sample.
//         The rotator is evaluated exactly at every kV-th sample and
//         advanced by that factor in between (at most kV - 1 products).
// Two spins per thread (one packed pair).
// ---------------------------------------------------------------------------
template <int S>
struct MSpins {
    static_assert(S % 2 == 0, "spins are processed in packed pairs");
    static constexpr int NP = S / 2;
    float xh[S], yh[S], zh[S], fh[S], vxh[S], vyh[S], vzh[S], m0[S], r1[S], r2[S];
    float mx[S], my[S], mz[S], em1[S], em2[S];
    int64_t base, end;
    int stride;
    float dt_cached;
    int rf_mode;
    // shared [7][S * stride]: lo halves of x, y, z, df, v_x, v_y, v_z of slot
    // s of thread t at t + s * stride (the kernel copies them once)
    const float* slo = nullptr;
    int sidx = 0;

    __device__ __forceinline__ float lo(int q, int s) const { return slo[q * (S * stride) + sidx + s * stride]; }

    __device__ __forceinline__ int64_t index(int s) const { return base + static_cast<int64_t>(s) * stride; }

    __device__ __forceinline__ void load(const float* __restrict__ P, const float* __restrict__ V, int64_t np,
                                         int64_t base_, int stride_, int64_t end_) {
        base = base_;
        stride = stride_;
        end = end_;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = index(s);
            const bool v = j < end;
            xh[s] = v ? P[P32_XH * np + j] : 0.f;
            yh[s] = v ? P[P32_YH * np + j] : 0.f;
            zh[s] = v ? P[P32_ZH * np + j] : 0.f;
            fh[s] = v ? P[P32_FH * np + j] : 0.f;
            m0[s] = v ? P[P32_M0 * np + j] : 0.f;
            r1[s] = v ? P[P32_R1 * np + j] : 0.f;
            r2[s] = v ? P[P32_R2 * np + j] : 0.f;
            vxh[s] = v ? V[PV32_XH * np + j] : 0.f;
            vyh[s] = v ? V[PV32_YH * np + j] : 0.f;
            vzh[s] = v ? V[PV32_ZH * np + j] : 0.f;
            mx[s] = 0.f;
            my[s] = 0.f;
            mz[s] = m0[s];
            em1[s] = 0.f;
            em2[s] = 0.f;
        }
        dt_cached = -1.f;
        rf_mode = 0;
    }

    // Rotation path of an RF run (header record): the field's z part
    // vanishes for every spin at every time (uniform rotation), or the
    // half angle stays <= 0.754 for every spin wherever it has moved by the
    // run's last midpoint (series path), else the general path.
    __device__ __forceinline__ void set_mode(const RecM& H, const float (&ext)[4], const float (&vext)[3]) {
        const float mb = H.a[7], mgx = H.a[8], mgy = H.a[9], mgz = H.a[10], mdt = H.a[11], tmax = H.a[12];
        const float ex = fmaf(vext[0], tmax, ext[0]), ey = fmaf(vext[1], tmax, ext[1]),
                    ez = fmaf(vext[2], tmax, ext[2]);
        const bool same = (mgx == 0.f || ex == 0.f) && (mgy == 0.f || ey == 0.f) && (mgz == 0.f || ez == 0.f) &&
                          ext[3] == 0.f;
        const float bound = mb + mgx * ex + mgy * ey + mgz * ez + mdt * 3.14159265358979323846f * ext[3];
        rf_mode = same ? (mb <= 0.754f ? 3 : 2) : (bound <= 0.754f ? 1 : 0);
    }

    // Rotate slot s by the quaternion (ch, u) (c2 = 2/|q|^2 to first order),
    // then relax over the step.
    __device__ __forceinline__ void rotate_relax(int s, float ch, float ux, float uy, float uz, float c2) {
        const float px = fmaf(uy, mz[s], -uz * my[s]);
        const float py = fmaf(uz, mx[s], -ux * mz[s]);
        const float pz = fmaf(ux, my[s], -uy * mx[s]);
        const float qx = fmaf(uy, pz, -uz * py);
        const float qy = fmaf(uz, px, -ux * pz);
        const float qz = fmaf(ux, py, -uy * px);
        const float nx = fmaf(c2, fmaf(ch, px, qx), mx[s]);
        const float ny = fmaf(c2, fmaf(ch, py, qy), my[s]);
        const float nz = fmaf(c2, fmaf(ch, pz, qz), mz[s]);
        mx[s] = fmaf(em2[s], nx, nx);
        my[s] = fmaf(em2[s], ny, ny);
        mz[s] = fmaf(em1[s], nz - m0[s], nz);
    }

    // One excitation step (quaternion w = cos|theta|, u = -theta sin|theta|/|theta|
    // of the half-angle vector theta, as in K1; cos and sinc as even series
    // in |theta|^2 on the SMALL path).
    template <bool SMALL>
    __device__ __forceinline__ void rf_slots(float gx, float gy, float gz, float bx, float by, float b2, float dt,
                                             float tm) {
        const float pdt = dt * 3.14159265358979323846f;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float px = fmaf(vxh[s], tm, xh[s]), py = fmaf(vyh[s], tm, yh[s]), pz = fmaf(vzh[s], tm, zh[s]);
            const float az = fmaf(gx, px, fmaf(gy, py, fmaf(gz, pz, fh[s] * pdt)));
            const float t2 = fmaf(az, az, b2);
            float ch, nsinc;
            if (SMALL) {
                float q = fmaf(t2, -2.75573192239858907e-6f, 1.98412698412698413e-4f);   // -1/9!, 1/7!
                q = fmaf(q, t2, -8.33333333333333333e-3f);                               // -1/5!
                q = fmaf(q, t2, 1.66666666666666667e-1f);                                // 1/3!
                nsinc = fmaf(q, t2, -1.0f);
                float c = fmaf(t2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);  // -1/10!, 1/8!
                c = fmaf(c, t2, -1.38888888888888889e-3f);                               // -1/6!
                c = fmaf(c, t2, 4.16666666666666667e-2f);                                // 1/4!
                c = fmaf(c, t2, -0.5f);
                ch = fmaf(c, t2, 1.0f);
            } else {
                const float rs = rsqrtf(t2);
                float sh;
                sincospi_f32(t2 * rs * 0.318309886183790671538f, &sh, &ch);
                nsinc = -sh * rs;
            }
            const float ux = bx * nsinc, uy = by * nsinc, uz = az * nsinc;
            const float nq = fmaf(ch, ch, fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
            rotate_relax(s, ch, ux, uy, uz, fmaf(-2.f, nq, 4.f));
        }
    }

    __device__ __forceinline__ void rf(const RecM& R, const float (&ext)[4], const float (&vext)[3]) {
        const float gx = R.a[0], gy = R.a[1], gz = R.a[2];
        const float bx = R.a[3], by = R.a[4], b2 = R.a[5], dt = R.a[6], tm = R.a[13];
        if (R.count > 0) set_mode(R, ext, vext);
        if (dt != dt_cached) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                em1[s] = expm1_f32(-dt * r1[s] * 0.693147180559945309f);
                em2[s] = expm1_f32(-dt * r2[s] * 0.693147180559945309f);
            }
            dt_cached = dt;
        }
        if (rf_mode >= 2) {
            float ch, f;
            if (rf_mode == 3) {
                float q = fmaf(b2, -2.75573192239858907e-6f, 1.98412698412698413e-4f);   // -1/9!, 1/7!
                q = fmaf(q, b2, -8.33333333333333333e-3f);                                       // -1/5!
                q = fmaf(q, b2, 1.66666666666666667e-1f);                                        // 1/3!
                f = fmaf(q, b2, -1.0f);
                float c = fmaf(b2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);  // -1/10!, 1/8!
                c = fmaf(c, b2, -1.38888888888888889e-3f);                                       // -1/6!
                c = fmaf(c, b2, 4.16666666666666667e-2f);                                        // 1/4!
                c = fmaf(c, b2, -0.5f);
                ch = fmaf(c, b2, 1.0f);
            } else {
                const float rs = rsqrtf(b2);
                float sh;
                sincospi_f32(b2 * rs * 0.318309886183790671538f, &sh, &ch);
                f = -sh * rs;
            }
            const float ux = bx * f, uy = by * f;
            const float c2 = fmaf(-2.f, fmaf(ch, ch, fmaf(ux, ux, uy * uy)), 4.f);
#pragma unroll
            for (int s = 0; s < S; ++s)
                rotate_relax(s, ch, ux, uy, 0.f, c2);
        } else if (rf_mode == 1) {
            rf_slots<true>(gx, gy, gz, bx, by, b2, dt, tm);
        } else {
            rf_slots<false>(gx, gy, gz, bx, by, b2, dt, tm);
        }
    }

    // Transverse magnetisation at (K, K1, tau) relative to t_ref:
    // Mxy(t_ref) e^{-tau/T2} e^{-i 2 pi (K.x + K1.v + df tau)}; hi/lo
    // products for every term (`koff`: where the record keeps K1).
    __device__ __forceinline__ void exact(const RecM& R, bool prec, int koff, const float* __restrict__ P,
                                          const float* __restrict__ V, int64_t np, int used, float (&er)[S],
                                          float (&ei)[S]) {
        const int terms = (R.count >> kTermShift) & used;
        const float th = R.a[6], tl = R.a[7];
        if (terms) {
            // the phase's terms, each a uniform branch around all slots
            float F[S];
#pragma unroll
            for (int s = 0; s < S; ++s) F[s] = 0.f;
            auto term = [&](int bit, const float (&ch)[S], int q, float kh, float kl) {
                if (terms & bit) {
#pragma unroll
                    for (int s = 0; s < S; ++s) F[s] += frac_product(ch[s], lo(q, s), kh, kl);
                }
            };
            term(1, xh, 0, R.a[0], R.a[1]);
            term(2, yh, 1, R.a[2], R.a[3]);
            term(4, zh, 2, R.a[4], R.a[5]);
            term(8, fh, 3, th, tl);
            term(16, vxh, 4, R.a[koff], R.a[koff + 1]);
            term(32, vyh, 5, R.a[koff + 2], R.a[koff + 3]);
            term(64, vzh, 6, R.a[koff + 4], R.a[koff + 5]);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float r = F[s] - rintf(F[s]);
                float sn, cs;
                __sincosf(-6.28318530717958647692f * r, &sn, &cs);
                const float e2 = exp2f(-th * r2[s]);
                er[s] = e2 * fmaf(mx[s], cs, -my[s] * sn);
                ei[s] = e2 * fmaf(mx[s], sn, my[s] * cs);
            }
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float e2 = exp2f(-th * r2[s]);
                er[s] = e2 * mx[s];
                ei[s] = e2 * my[s];
            }
        }
        if (prec) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float e1 = exp2f(-th * r1[s]);
                mx[s] = er[s];
                my[s] = ei[s];
                mz[s] = fmaf(mz[s] - m0[s], e1, m0[s]);
            }
        }
    }

    // ADC record of L samples from (er, ei); sink(i, re, im) gets the warp
    // sums of sample i on one lane.
    template <class Sink>
    __device__ __forceinline__ void adc(const RecM& R, int L, const float* __restrict__ V, int64_t np, int used,
                                        float (&er)[S], float (&ei)[S], int lane, Sink&& sink) {
        if (L == 1) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                sr += er[s];
                si += ei[s];
            }
            sr = warp_sum(sr);
            si = warp_sum(si);
            if (lane == 0) sink(0, sr, si);
            return;
        }
        const float dkx = R.a[8], dky = R.a[9], dkz = R.a[10], dtau = R.a[11];
        // the increment's linear term exists iff the gradient moves a moving spin
        const bool quad = (dkx != 0.f && (used & 16)) || (dky != 0.f && (used & 32)) || (dkz != 0.f && (used & 64));
        float phi1[S], phi2[S], mag[S];
        f32x2 wr[NP], wi[NP], wn[NP];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int64_t j = index(s);
            const bool v = j < end;
            float p = fmaf(dkx, xh[s], fmaf(dky, yh[s], fmaf(dkz, zh[s], fh[s] * dtau)));
            if (used & 16) p += frac_product(vxh[s], lo(4, s), R.a[18], R.a[19]);
            if (used & 32) p += frac_product(vyh[s], lo(5, s), R.a[20], R.a[21]);
            if (used & 64) p += frac_product(vzh[s], lo(6, s), R.a[22], R.a[23]);
            phi1[s] = p - rintf(p);
            phi2[s] = dtau * fmaf(dkx, vxh[s], fmaf(dky, vyh[s], dkz * vzh[s]));
            mag[s] = exp2f(-dtau * r2[s]);
        }
        if (quad) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float s0, c0, s1, c1;
                sincospi_f32(-2.f * phi2[2 * p], &s0, &c0);
                sincospi_f32(-2.f * phi2[2 * p + 1], &s1, &c1);
                wr[p] = pk(c0, c1);
                wi[p] = pk(s0, s1);
                wn[p] = pk(-s0, -s1);
            }
        }
        f32x2 pr[NP], pi_[NP], qr[NP], qi[NP], qn[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            pr[p] = pk(er[2 * p], er[2 * p + 1]);
            pi_[p] = pk(ei[2 * p], ei[2 * p + 1]);
        }
        for (int c = 0; c < L; c += kV) {
            if (c == 0 || quad) {
                // rotator of sample c exactly: mag e^{-i 2 pi (phi1 + c phi2)}
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    float zs[2], zc[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int s = 2 * p + h;
                        float q = fmaf(static_cast<float>(c), phi2[s], phi1[s]);
                        q -= rintf(q);
                        sincospi_f32(-2.f * q, &zs[h], &zc[h]);
                        zs[h] *= mag[s];
                        zc[h] *= mag[s];
                    }
                    qr[p] = pk(zc[0], zc[1]);
                    qi[p] = pk(zs[0], zs[1]);
                    qn[p] = pk(-zs[0], -zs[1]);
                }
            }
            float ar[kV], ai[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                f32x2 sr2 = pr[0], si2 = pi_[0];
#pragma unroll
                for (int p = 1; p < NP; ++p) {
                    sr2 = add2(sr2, pr[p]);
                    si2 = add2(si2, pi_[p]);
                }
                float r0, r1_, i0, i1;
                unpk(sr2, r0, r1_);
                unpk(si2, i0, i1);
                ar[v] = r0 + r1_;
                ai[v] = i0 + i1;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const f32x2 nr2 = fma2(pr[p], qr[p], mul2(pi_[p], qn[p]));
                    pi_[p] = fma2(pr[p], qi[p], mul2(pi_[p], qr[p]));
                    pr[p] = nr2;
                    if (quad) {
                        const f32x2 zr2 = fma2(qr[p], wr[p], mul2(qi[p], wn[p]));
                        qi[p] = fma2(qr[p], wi[p], mul2(qi[p], wr[p]));
                        qr[p] = zr2;
                        qn[p] = neg2(qi[p]);
                    }
                }
            }
            const float sr = reduce_scatter8(ar, lane);
            const float si = reduce_scatter8(ai, lane);
            const int vl = (lane >> 2) & 7;
            if ((lane & 3) == 0 && c + vl < L) sink(c + vl, sr, si);
        }
    }
};

template <int S, bool SPLIT>
__global__ void __launch_bounds__(kMaxBlock, 2) bloch_motion_kernel(const __grid_constant__ BlochArgs A) {
    __shared__ __align__(128) RecM s_rec[2][kTile];
    __shared__ __align__(8) uint64_t s_bar[2];
    extern __shared__ __align__(16) float2 s_red_dyn[];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nthr = blockDim.x;
    const int nwarps = nthr >> 5;
    const int cta = blockIdx.x;
    // ADC-run split: CTAs cta = spin_cta * split + part share one spin range;
    // part p handles the ADC records whose index is p mod split
    const int split = SPLIT ? A.split : 1;
    const int part = SPLIT ? cta % split : 0, scta = SPLIT ? cta / split : cta;

    int64_t c_begin, c_end;
    if (A.cta_begin) {
        c_begin = A.cta_begin[scta];
        c_end = A.cta_begin[scta + 1];
    } else {
        c_begin = static_cast<int64_t>(scta) * A.spins_per_cta;
        c_end = min(A.n, c_begin + A.spins_per_cta);
    }
    const int64_t np = A.n_pad;
    MSpins<S> sp;
    sp.load(A.p32, A.pv32, np, c_begin + tid, nthr, c_end);
    // the lo halves of the CTA's positions, off-resonances and velocities,
    // in dynamic shared memory after the reduction stage
    float* s_lo = reinterpret_cast<float*>(s_red_dyn + 2 * nwarps * kRed32);
    for (int i = tid; i < S * nthr; i += nthr) {
        const int64_t j = c_begin + i;
        const bool v = j < c_end;
        s_lo[0 * S * nthr + i] = v ? A.p32[P32_XL * np + j] : 0.f;
        s_lo[1 * S * nthr + i] = v ? A.p32[P32_YL * np + j] : 0.f;
        s_lo[2 * S * nthr + i] = v ? A.p32[P32_ZL * np + j] : 0.f;
        s_lo[3 * S * nthr + i] = v ? A.p32[P32_FL * np + j] : 0.f;
        s_lo[4 * S * nthr + i] = v ? A.pv32[PV32_XL * np + j] : 0.f;
        s_lo[5 * S * nthr + i] = v ? A.pv32[PV32_YL * np + j] : 0.f;
        s_lo[6 * S * nthr + i] = v ? A.pv32[PV32_ZL * np + j] : 0.f;
    }
    sp.slo = s_lo;
    sp.sidx = tid;

    int red_buf = 0;
    int64_t red_base = 0, red_end = 0;  // samples [red_base, red_end) staged
    // one partial row per spin range; with a split each part writes the
    // samples of its own runs (s_own marks them in the staged window)
    __shared__ unsigned char s_own[SPLIT ? 2 : 1][SPLIT ? kRed32 : 1];
    float2* __restrict__ partial = static_cast<float2*>(A.partial) + static_cast<int64_t>(scta) * A.n_adc;
    auto red_slot = [&](int buf, int w, int i) -> float2& { return s_red_dyn[(buf * nwarps + w) * kRed32 + i]; };
    auto flush = [&]() {
        __syncthreads();
        const int cnt = static_cast<int>(red_end - red_base);
        for (int i = tid; i < cnt; i += nthr) {
            if (SPLIT && !s_own[red_buf][i]) continue;
            // the warps' sums added by TwoSum: the CTA's total is rounded once
            TwoSumAcc sr, si;
            for (int w = 0; w < nwarps; ++w) {
                const float2 v = red_slot(red_buf, w, i);
                sr.add(v.x);
                si.add(v.y);
            }
            partial[red_base + i] = make_float2(sr.value32(), si.value32());
        }
        red_buf ^= 1;
        red_base = red_end;
    };

    const BarPair bar{smem_u32(&s_bar[0])};
    const RecM* __restrict__ grec = static_cast<const RecM*>(A.rec);
    const int64_t n_tiles = (A.n_rec + kTile - 1) / kTile;
    auto issue = [&](int64_t t) {
        const int64_t nr = min(static_cast<int64_t>(kTile), A.n_rec - t * kTile);
        tma_load_1d(smem_u32(&s_rec[t & 1][0]), grec + t * kTile, static_cast<uint32_t>(nr * sizeof(RecM)),
                    bar[t & 1]);
    };
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int64_t t = 0; t < 2 && t < n_tiles; ++t) issue(t);
    }

    for (int64_t t = 0; t < n_tiles; ++t) {
        const int b = static_cast<int>(t & 1);
        const bool ok = mbar_wait_bounded(bar[b], static_cast<uint32_t>((t >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(A.status, kStatusTimeout);
                mbar_wait_bounded(bar[b], static_cast<uint32_t>((t >> 1) & 1));
                if (t + 1 < n_tiles) mbar_wait_bounded(bar[b ^ 1], static_cast<uint32_t>(((t + 1) >> 1) & 1));
            }
            return;
        }
        const int nr = static_cast<int>(min(static_cast<int64_t>(kTile), A.n_rec - t * kTile));
        for (int r = 0; r < nr; ++r) {
            const RecM& R = s_rec[b][r];
            const int type = R.type;
            if (type == REC_RF) {
                sp.rf(R, A.ext, A.vext);
            } else if (type == REC_PREC) {
                float er[S], ei[S];
                sp.exact(R, true, 8, A.p32, A.pv32, np, A.used, er, ei);
            } else if (type == REC_ADC) {
                const int L = min(max(R.count & kCountMask, 1), kMaxAdcRun);
                const int64_t k0 = R.k0;
                if (k0 < red_base || k0 + L > A.n_adc) {  // inside the row, not before the staged window
                    if (tid == 0) atomicOr(A.status, kStatusBadAdc);
                    continue;
                }
                if (k0 + L > red_base + kRed32) flush();
                const int off = static_cast<int>(k0 - red_base);
                const bool own = !SPLIT || (t * kTile + r) % split == part;
                if (SPLIT && warp == 0)
                    for (int i = lane; i < L; i += 32) s_own[red_buf][off + i] = own;
                if (own) {
                    float er[S], ei[S];
                    sp.exact(R, false, 12, A.p32, A.pv32, np, A.used, er, ei);
                    sp.adc(R, L, A.pv32, np, A.used, er, ei, lane,
                           [&](int i, float sr, float si) { red_slot(red_buf, warp, off + i) = make_float2(sr, si); });
                }
                red_end = k0 + L;
            }
        }
        __syncthreads();  // everyone is done with tile buffer b
        if (tid == 0 && t + 2 < n_tiles) {
            fence_proxy_async_smem();
            issue(t + 2);
        }
    }
    if (red_end > red_base) flush();
}

// ---------------------------------------------------------------------------
// K1d: FP64 Bloch kernel (one spin per thread, every sample evaluated exactly).
// Records are read from global memory (uniform addresses, L1 broadcast).
// MOV: the spin moves, x(t) = x + v t: an RF step sees the position at its
// midpoint t_mid, and a phase from t_ref to t is 2 pi (K.x + K1.v + df tau)
// with K1 of sample l of a run equal to K1 + l dK1_0 + l (l - 1) / 2 dtau dK.
// ---------------------------------------------------------------------------
template <bool MOV>
__global__ void __launch_bounds__(kMaxBlock) bloch_fp64_kernel(const __grid_constant__ BlochArgs A) {
    __shared__ __align__(16) double2 s_red[2][kMaxWarps][kRed];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nthr = blockDim.x;
    const int nwarps = nthr >> 5;
    const int cta = blockIdx.x;
    int64_t c_begin, c_end;
    if (A.cta_begin) {
        c_begin = A.cta_begin[cta];
        c_end = A.cta_begin[cta + 1];
    } else {
        c_begin = static_cast<int64_t>(cta) * A.spins_per_cta;
        c_end = min(A.n, c_begin + A.spins_per_cta);
    }
    const int64_t j = c_begin + tid;
    const bool v = j < c_end;
    const int64_t np = A.n_pad;
    const double* __restrict__ P = A.p64;
    const double x = v ? P[P64_X * np + j] : 0.0;
    const double y = v ? P[P64_Y * np + j] : 0.0;
    const double z = v ? P[P64_Z * np + j] : 0.0;
    const double f = v ? P[P64_F * np + j] : 0.0;
    const double T1 = v ? P[P64_T1 * np + j] : 1.0;
    const double T2 = v ? P[P64_T2 * np + j] : 1.0;
    const double m0 = v ? P[P64_M0 * np + j] : 0.0;
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (MOV && v) {
        vx = A.pv64[j];
        vy = A.pv64[np + j];
        vz = A.pv64[2 * np + j];
    }
    double mx = 0.0, my = 0.0, mz = m0, em1 = 0.0, em2 = 0.0, dt_cached = -1.0;

    int red_buf = 0;
    int64_t red_base = 0, red_end = 0;
    double2* __restrict__ partial = static_cast<double2*>(A.partial) + static_cast<int64_t>(cta) * A.n_adc;
    auto flush = [&]() {
        __syncthreads();
        const int cnt = static_cast<int>(red_end - red_base);
        for (int i = tid; i < cnt; i += nthr) {
            double sr = 0.0, si = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                const double2 q = s_red[red_buf][w][i];
                sr += q.x;
                si += q.y;
            }
            partial[red_base + i] = make_double2(sr, si);
        }
        red_buf ^= 1;
        red_base = red_end;
    };

    const Rec64* __restrict__ rec = static_cast<const Rec64*>(A.rec);
    for (int64_t r = 0; r < A.n_rec; ++r) {
        const Rec64& R = rec[r];
        const int type = R.type;
        if (type == REC_RF) {
            const double gx = R.a[0], gy = R.a[1], gz = R.a[2], bx = R.a[3], by = R.a[4], dt = R.a[5];
            if (dt != dt_cached) {
                em1 = expm1(-dt / T1);
                em2 = expm1(-dt / T2);
                dt_cached = dt;
            }
            double px0 = x, py0 = y, pz0 = z;
            if (MOV) {
                const double tm = R.a[6];
                px0 = fma(vx, tm, x);
                py0 = fma(vy, tm, y);
                pz0 = fma(vz, tm, z);
            }
            const double az = gx * px0 + gy * py0 + gz * pz0 + f * dt;
            const double an = sqrt(bx * bx + by * by + az * az);
            double sh, ch;
            sincospi(an, &sh, &ch);
            const double fct = an > 0.0 ? -sh / an : 0.0;
            const double ux = bx * fct, uy = by * fct, uz = az * fct;
            const double px = uy * mz - uz * my, py = uz * mx - ux * mz, pz = ux * my - uy * mx;
            const double qx = uy * pz - uz * py, qy = uz * px - ux * pz, qz = ux * py - uy * px;
            const double nx = mx + 2.0 * (ch * px + qx);
            const double ny = my + 2.0 * (ch * py + qy);
            const double nz = mz + 2.0 * (ch * pz + qz);
            mx = nx + em2 * nx;
            my = ny + em2 * ny;
            mz = nz + em1 * (nz - m0);
        } else if (type == REC_PREC) {
            double F = R.a[0] * x + R.a[1] * y + R.a[2] * z + f * R.a[3];
            if (MOV) F += R.a[4] * vx + R.a[5] * vy + R.a[6] * vz;
            double sn, cs;
            sincospi(-2.0 * F, &sn, &cs);
            const double e2 = exp(-R.a[3] / T2), e1 = exp(-R.a[3] / T1);
            const double nx = e2 * (mx * cs - my * sn);
            const double ny = e2 * (mx * sn + my * cs);
            mx = nx;
            my = ny;
            mz = m0 + (mz - m0) * e1;
        } else if (type == REC_ADC) {
            const int L = min(max(R.count, 1), kMaxAdcRun);
            const int64_t k0 = R.k0;
            if (k0 < red_base || k0 + L > A.n_adc) {  // inside the row, not before the staged window
                if (threadIdx.x == 0) atomicOr(A.status, kStatusBadAdc);
                continue;
            }
            if (k0 + L > red_base + kRed) flush();
            for (int l = 0; l < L; ++l) {
                const double kx = R.a[0] + l * R.a[4], ky = R.a[1] + l * R.a[5], kz = R.a[2] + l * R.a[6];
                const double tau = R.a[3] + l * R.a[7];
                double F = kx * x + ky * y + kz * z + f * tau;
                if (MOV) {
                    const double c2 = 0.5 * l * (l - 1) * R.a[7];
                    const double k1x = R.a[8] + l * R.a[11] + c2 * R.a[4];
                    const double k1y = R.a[9] + l * R.a[12] + c2 * R.a[5];
                    const double k1z = R.a[10] + l * R.a[13] + c2 * R.a[6];
                    F += k1x * vx + k1y * vy + k1z * vz;
                }
                double sn, cs;
                sincospi(-2.0 * F, &sn, &cs);
                const double e2 = v ? exp(-tau / T2) : 0.0;
                double sr = warp_sum(e2 * (mx * cs - my * sn));
                double si = warp_sum(e2 * (mx * sn + my * cs));
                if (lane == 0) s_red[red_buf][warp][k0 + l - red_base] = make_double2(sr, si);
            }
            red_end = k0 + L;
        }
    }
    if (red_end > red_base) flush();
}

// ---------------------------------------------------------------------------
// K6: tensor-core readout (the matrix form of a group of ADC runs).
//
// For a group of R <= 64 runs sharing the rotator z_s and a block of 32
// spins, the signal contribution is the complex product
//   C[r][l] = sum_s E_s(r) z_s^l
// written as one real product of a 128-row matrix (rows 2r, 2r+1 = Re, Im of
// run r) by the 128 samples: with k = (spin s, part p) the contraction index,
//   A[2r][s,0] = Re E   A[2r][s,1] = -Im E   A[2r+1][s,0] = Im E   A[2r+1][s,1] = Re E
//   B[l][s,0]  = Re z^l B[l][s,1]  = Im z^l
// so D = A B^T holds Re C in row 2r and Im C in row 2r+1. Operands are FP16
// pairs hi + lo (hi = fp16(v), lo = fp16(v - hi)): the three products
// hi hi + hi lo + lo hi carry ~22 bits, accumulated in FP32 in tensor memory
// across every spin block of the CTA. One tcgen05.mma (kind::f16, M = N =
// 128, K = 16) takes 8 spins; a 32-spin block is 4 x 3 of them.
//
// Pipeline per CTA (one per SM), warp-specialised, block i of the flattened
// (group, block) sequence:
//   16 E warps, once the MMAs of block i - 2 have released stage i & 1
//   ("empty", the tensor core's commit), copy block i + 2's snapshot rows
//   and spin parameters into staging buffer (i + 2) % 4 with cp.async (that
//   buffer held block i - 2, whose fill preceded those MMAs); each thread
//   arrives on "staged" when its copies have landed; they then turn block
//   i's staging into the E operand slices of stage i & 1 and arrive on
//   "full";
//   8 B warps wait for the same "empty" and "staged", write the rotator
//   slices of stage i & 1 and arrive on "full";
//   one MMA warp waits for "full", issues block i's 12 MMAs into accumulator
//   buffer (segment & 1) and commits them to "empty" (a group's blocks form
//   segments of kMmaSegBlocks, numbered across groups);
//   after a segment's last block the E warps read its accumulator from
//   tensor memory and release the buffer ("accumulator read"): they add it
//   into the group's running sum, kept in tensor memory as an FP32 pair
//   (sum, error) by TwoSum, and after the group's last segment write the
//   compensated total into the CTA's partial row. The FP32 accumulation of
//   the tensor core thus runs over at most 12 kMmaSegBlocks products per
//   element, and the sum over segments is exact up to its final rounding.
// Every wait is bounded; a wait that gives up stops every role.
// Operand slices: 128 rows x 16 FP16 (4 KB), K-major without swizzle: 8-row
// x 16-byte core matrices, K-adjacent ones 128 B apart, row-adjacent ones
// 256 B apart. z_s^l comes from z^(j + 64 g) and z^8 (direct, with an exact
// phase reduction) and seven complex products: l = 64 g + 8 q + j.
// ---------------------------------------------------------------------------
constexpr int kMmaThreads = 512;                    // E-slice producer threads (16 warps)
constexpr int kMmaZThreads = 256;                   // B-slice producer threads (8 warps)
constexpr int kMmaCtaThreads = kMmaThreads + kMmaZThreads + 32;  // + the MMA warp
constexpr int kMmaChunk = 32;                       // spins per block
constexpr int kMmaTileBytes = 128 * 16 * 2;         // one K = 16 slice of a 128-row FP16 operand
constexpr int kMmaStageBytes = 16 * kMmaTileBytes;  // A hi, A lo, B hi, B lo x 4 slices (64 KB)
constexpr int kMmaERowBytes = kMmaChunk * 8 + 32;   // staged snapshot row: 32 spins + 32 B (bank spread)
constexpr int kMmaStageE = kMmaRuns * kMmaERowBytes;           // 18 KB
// + the block's xh, xl, yh, yl, zh, zl, fh, fl, r2 (staged in this order)
constexpr int kMmaParams = 9;
constexpr int kMmaStageIn = kMmaStageE + kMmaParams * kMmaChunk * 4;
constexpr int kMmaStageInPad = (kMmaStageIn + 127) / 128 * 128;
constexpr int kMmaStaging = 4;                      // staging buffers (the loader runs up to 4 blocks ahead)
// Tensor memory: two FP32 accumulators of 128 lanes x 128 columns (the MMAs
// of one segment of kMmaSegBlocks blocks go into one while the other is
// drained), then the group's running sum of its drained segments as an
// unevaluated FP32 pair (sum, error) of 128 columns each.
constexpr uint32_t kMmaTmemCols = 512;
constexpr uint32_t kMmaSumCol = 256;                // running sum of the group
constexpr uint32_t kMmaErrCol = 384;                // its accumulated rounding errors
constexpr int kMmaSegBlocks = 8;                    // blocks accumulated in FP32 before a drain
constexpr size_t kMmaDynSmem = 2 * kMmaStageBytes + kMmaStaging * kMmaStageInPad + 256;  // one CTA per SM

// byte offset of the 16-byte row word (row, K group kg of 8 elements) in a slice
__device__ __forceinline__ uint32_t mma_word_off(int row, int kg) {
    return static_cast<uint32_t>((row >> 3) * 256 + kg * 128 + (row & 7) * 16);
}
// shared-memory matrix descriptor: start address, leading (K) byte offset
// 128, stride (row) byte offset 256, in 16-byte units; bits 46..48 = 0b001
// (the tcgen05 descriptor version); no swizzle
__device__ __forceinline__ uint64_t mma_smem_desc(uint32_t addr) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(128 >> 4) << 16) |
           (static_cast<uint64_t>(256 >> 4) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: D FP32, A and B FP16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kMmaIdesc = (1u << 4) | (static_cast<uint32_t>(128 >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kMmaIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// 16 FP32 columns of this warp's 32 TMEM lanes (lane quarter warp % 4)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 4 FP32 columns of this warp's 32 TMEM lanes: load and store, completed by
// tc_wait_ld / tc_wait_st (several in flight behind one wait)
__device__ __forceinline__ void tc_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_st4(uint32_t taddr, const float (&v)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3]))
                 : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// v = hi + lo as FP16 pairs (a in the low half)
__device__ __forceinline__ void split_half2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// 2^x (PTX ex2.approx, subnormal results flushed to zero: the decays here
// are factors in (0, 1] next to unit-scale values)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// two complex values (re, im: one spin per half) split into FP16 hi + lo
// words, one word per spin: (re, im) with re in the low half
__device__ __forceinline__ void split_cplx2(f32x2 re, f32x2 im, uint32_t (&hi)[2], uint32_t (&lo)[2]) {
    float r0, r1, i0, i1;
    unpk(re, r0, r1);
    unpk(im, i0, i1);
    const __half2 h0 = __floats2half2_rn(r0, i0), h1 = __floats2half2_rn(r1, i1);
    const f32x2 lr = sub2(re, pk(__low2float(h0), __low2float(h1)));
    const f32x2 li = sub2(im, pk(__high2float(h0), __high2float(h1)));
    float a0, a1, b0, b1;
    unpk(lr, a0, a1);
    unpk(li, b0, b1);
    const __half2 l0 = __floats2half2_rn(a0, b0), l1 = __floats2half2_rn(a1, b1);
    hi[0] = *reinterpret_cast<const uint32_t*>(&h0);
    hi[1] = *reinterpret_cast<const uint32_t*>(&h1);
    lo[0] = *reinterpret_cast<const uint32_t*>(&l0);
    lo[1] = *reinterpret_cast<const uint32_t*>(&l1);
}

// Constants of one run of the E slices, both halves equal (built once per
// group): K0 hi/lo per axis, tau0 hi/lo, -tau0
struct MmaRunPk {
    f32x2 kh[3], kl[3], th, tl, nth;
    __device__ __forceinline__ void set(const MmaRun& r) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            kh[d] = bcast2(r.kh[d]);
            kl[d] = bcast2(r.kl[d]);
        }
        th = bcast2(r.th);
        tl = bcast2(r.tl);
        nth = bcast2(-r.th);
    }
};
// Constants of one group's rotator, both halves equal: -dK, -dtau, dtau
struct MmaGroupPk {
    f32x2 ndk[3], ndtau, dtau;
    __device__ __forceinline__ void set(const MmaGroup& g) {
#pragma unroll
        for (int d = 0; d < 3; ++d) ndk[d] = bcast2(-g.dk[d]);
        ndtau = bcast2(-g.dtau);
        dtau = bcast2(g.dtau);
    }
};

// A slices (E part) of a stage: thread = (run r, spin quad); it evaluates
// E_s(r) = Mxy_s(t_ref) e^{-tau0/T2} e^{-i 2 pi (K0.x + df tau0)} for its 4
// spins, two at a time (the Bloch kernel's exact evaluation: hi/lo phase
// products, exact reduction to a fractional turn, hardware sine) and writes
// rows 2r (Re E, -Im E) and 2r + 1 (Im E, Re E), hi and lo. Runs past n_runs
// and spins past the block's `live` ones give zero rows. The x and y terms
// are always formed (a zero factor gives a zero term), the z and
// off-resonance terms only when some spin has them (kZ, kDF): no branches in
// the phase chain.
template <bool kZ, bool kDF>
__device__ __forceinline__ void mma_fill_e(unsigned char* stage, const unsigned char* in, const MmaRunPk& run,
                                           bool run_live, bool one_snap, int live, int warp, int lane) {
    const int r = 4 * warp + (lane & 3), q8 = lane >> 2;
    const int kap = q8 >> 1, kg = q8 & 1, sb = 8 * kap + 4 * kg;
    constexpr int R = kMmaChunk / 2;  // pairs per staged parameter row
    f32x2 er[2] = {0ull, 0ull}, nei[2] = {0ull, 0ull};
    if (run_live) {
        const f32x2* prm = reinterpret_cast<const f32x2*>(in + kMmaStageE) + (sb >> 1);
        const float4* m4 = reinterpret_cast<const float4*>(in + (one_snap ? 0 : r) * kMmaERowBytes + sb * 8);
        const float4 ma = m4[0], mb = m4[1];
        const float mx[4] = {ma.x, ma.z, mb.x, mb.z}, my[4] = {ma.y, ma.w, mb.y, mb.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f32x2* q = prm + h;
            f32x2 F = add2(frac_product2(q[0 * R], q[1 * R], run.kh[0], run.kl[0]),
                           frac_product2(q[2 * R], q[3 * R], run.kh[1], run.kl[1]));
            if (kZ) F = add2(F, frac_product2(q[4 * R], q[5 * R], run.kh[2], run.kl[2]));
            if (kDF) F = add2(F, frac_product2(q[6 * R], q[7 * R], run.th, run.tl));
            float a0, a1, d0, d1, s0, c0, s1, c1;
            unpk(mul2(frac2(F), bcast2(-6.28318530717958647692f)), a0, a1);
            __sincosf(a0, &s0, &c0);
            __sincosf(a1, &s1, &c1);
            unpk(mul2(run.nth, q[8 * R]), d0, d1);
            const float e0 = ex2_approx(d0), e1 = ex2_approx(d1);
            const int i0 = 2 * h, i1 = 2 * h + 1;
            const bool v0 = sb + i0 < live, v1 = sb + i1 < live;
            er[h] = pk(v0 ? e0 * fmaf(mx[i0], c0, -my[i0] * s0) : 0.f, v1 ? e1 * fmaf(mx[i1], c1, -my[i1] * s1) : 0.f);
            nei[h] = pk(v0 ? -e0 * fmaf(mx[i0], s0, my[i0] * c0) : 0.f, v1 ? -e1 * fmaf(mx[i1], s1, my[i1] * c1) : 0.f);
        }
    }
    uint32_t hi[4], lo[4], hi2[4], lo2[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t a[2], b[2];
        split_cplx2(er[h], nei[h], a, b);
        hi[2 * h] = a[0];
        hi[2 * h + 1] = a[1];
        lo[2 * h] = b[0];
        lo[2 * h + 1] = b[1];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // (Im E, Re E): the halves swapped, the new low half negated (exact)
        hi2[q] = __byte_perm(hi[q], 0u, 0x1032) ^ 0x8000u;
        lo2[q] = __byte_perm(lo[q], 0u, 0x1032) ^ 0x8000u;
    }
    const uint32_t off = static_cast<uint32_t>(kap * kMmaTileBytes) + mma_word_off(2 * r, kg);
    *reinterpret_cast<uint4*>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(stage + 4 * kMmaTileBytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(stage + off + 16) = make_uint4(hi2[0], hi2[1], hi2[2], hi2[3]);
    *reinterpret_cast<uint4*>(stage + 4 * kMmaTileBytes + off + 16) = make_uint4(lo2[0], lo2[1], lo2[2], lo2[3]);
}

// B slices (rotator powers) of a stage, by the 8 B-slice warps: thread =
// (spin pair, j = l mod 8, g = l div 64), warp v: K slice v & 3, g = v >> 2;
// lane: pair half, j, K group. 2 spins (one per f32x2 half) x samples
// l = 64 g + 8 q + j, q < 8; a warp's 8-byte stores of one q fill 256
// contiguous bytes. Spins past the last one have zero parameters (z = 1) and
// zero E.
__device__ __forceinline__ void mma_fill_z(unsigned char* stage, const unsigned char* in, const MmaGroupPk& G,
                                           int v, int lane) {
    constexpr int NQ = 8;
    const int kap = v & 3, g = v >> 2;
    const int half = lane & 1, j = (lane >> 1) & 7, kg = lane >> 4;
    const int s2 = 8 * kap + 4 * kg + 2 * half;
    constexpr int R = kMmaChunk / 2;
    const f32x2* prm = reinterpret_cast<const f32x2*>(in + kMmaStageE) + (s2 >> 1);
    const f32x2 X = prm[0 * R], Y = prm[2 * R], Z = prm[4 * R], F = prm[6 * R], R2 = prm[8 * R];
    // turns per sample, as the Bloch kernel's rotator (the negated constants
    // give the same roundings as negating the sum)
    const f32x2 th1 = fma2(G.ndk[0], X, fma2(G.ndk[1], Y, fma2(G.ndk[2], Z, mul2(F, G.ndtau))));
    const f32x2 rate = mul2(G.dtau, R2);
    const float m0 = static_cast<float>(j + 8 * NQ * g);
    // one-shot phases (not accumulated beyond three products): the
    // fractional turn exactly reduced, then the hardware sine; 8 th1 is exact
    const f32x2 M0 = bcast2(m0);
    const f32x2 p = mul2(M0, th1);
    const f32x2 ph0 = add2(frac2(p), fma2(M0, th1, neg2(p)));
    const f32x2 ph8 = frac2(mul2(bcast2(8.f), th1));
    const f32x2 two_pi = bcast2(6.28318530717958647692f);
    float a0, a1, b0, b1, c0, s0, c1, s1, c8, s8, c9, s9;
    unpk(mul2(two_pi, ph0), a0, a1);
    unpk(mul2(two_pi, ph8), b0, b1);
    __sincosf(a0, &s0, &c0);
    __sincosf(a1, &s1, &c1);
    __sincosf(b0, &s8, &c8);
    __sincosf(b1, &s9, &c9);
    float d0, d1, e0, e1;
    unpk(mul2(bcast2(-m0), rate), d0, d1);
    unpk(mul2(bcast2(-8.f), rate), e0, e1);
    const f32x2 mag = pk(ex2_approx(d0), ex2_approx(d1)), mag8 = pk(ex2_approx(e0), ex2_approx(e1));
    f32x2 zr = mul2(mag, pk(c0, c1)), zi = mul2(mag, pk(s0, s1));
    const f32x2 wr = mul2(mag8, pk(c8, c9)), wi = mul2(mag8, pk(s8, s9)), nwi = neg2(wi);
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) {
        const int l = 8 * NQ * g + 8 * qq + j;
        uint32_t hi[2], lo[2];
        split_cplx2(zr, zi, hi, lo);
        const uint32_t off = static_cast<uint32_t>((8 + kap) * kMmaTileBytes) + mma_word_off(l, kg) + 8u * half;
        *reinterpret_cast<uint2*>(stage + off) = make_uint2(hi[0], hi[1]);
        *reinterpret_cast<uint2*>(stage + 4 * kMmaTileBytes + off) = make_uint2(lo[0], lo[1]);
        if (qq < NQ - 1) {
            const f32x2 nr = fma2(zr, wr, mul2(zi, nwi));
            zi = fma2(zr, wi, mul2(zi, wr));
            zr = nr;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Staging of one block by the 512 producer threads: the snapshot rows of
// the block's group (thread t copies 16 bytes of rows t / 16 and t / 16 + 32:
// the rows of the group's runs, or row 0 alone when they share one) and the
// block's spin parameters (threads 0..71). Spins past the last one are copied
// as they are (inside the padded rows) and read as zero. Each thread keeps its
// source rows (at spin 0) and destinations, set once per group, so a block
// costs it one 64-bit add and one cp.async per copy.
struct MmaStager {
    int group = -1;
    const float2* row[2] = {nullptr, nullptr};  // this thread's snapshot rows at spin 0 (+ its 16 bytes)
    bool has_row[2] = {false, false};
    const float* prm = nullptr;                 // its parameter row at spin 0 (+ its 16 bytes), threads < 72
    uint32_t dst_row = 0, dst_prm = 0;          // offsets in a staging buffer

    __device__ __forceinline__ void stage(uint32_t buf, const MmaArgs& A, int g, int64_t s0, int tid);
};

// 16-byte global -> shared copy (cp.async, L2 only), and the arrival on
// `bar` of this thread once all its earlier copies have landed
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void MmaStager::stage(uint32_t buf, const MmaArgs& A, int g, int64_t s0, int tid) {
    if (g != group) {
        const MmaGroup G = A.groups[g];
        const int rows = G.one_snap ? 1 : G.n_runs;
        const int q = tid & 15;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = (tid >> 4) + 32 * i;
            has_row[i] = r < rows;
            row[i] = has_row[i] ? A.snap + static_cast<int64_t>(A.runs[G.run0 + r].snap) * A.n_pad + 2 * q : nullptr;
        }
        dst_row = static_cast<uint32_t>((tid >> 4) * kMmaERowBytes + q * 16);
        if (group < 0 && tid < kMmaParams * 8) {
            const int a = tid >> 3, qq = tid & 7;
            const int prow = a == 0 ? P32_XH : a == 1 ? P32_XL : a == 2 ? P32_YH : a == 3 ? P32_YL : a == 4 ? P32_ZH
                           : a == 5 ? P32_ZL : a == 6 ? P32_FH : a == 7 ? P32_FL : P32_R2;
            prm = A.p32 + static_cast<int64_t>(prow) * A.n_pad + 4 * qq;
            dst_prm = static_cast<uint32_t>(kMmaStageE + a * kMmaChunk * 4 + qq * 16);
        }
        group = g;
    }
    if (has_row[0]) cp_async16(buf + dst_row, row[0] + s0);
    if (has_row[1]) cp_async16(buf + dst_row + 32 * kMmaERowBytes, row[1] + s0);
    if (prm != nullptr) cp_async16(buf + dst_prm, prm + s0);
}

template <bool kZ, bool kDF>
__global__ void __launch_bounds__(kMmaCtaThreads, 1) readout_mma_kernel(const __grid_constant__ MmaArgs A) {
    extern __shared__ __align__(1024) unsigned char s_mma[];
    unsigned char* s_in = s_mma + 2 * kMmaStageBytes;  // kMmaStaging staging buffers
    // mbarriers: [0, 1] stage full (producer threads arrive), [2, 3] stage
    // empty (MMA commit), [4, 5] accumulator buffer read (producer threads),
    // [6 .. 9] staging loaded (producer threads, on their copies' completion);
    // then the TMEM address, the abort flag, the commit count. A staging
    // buffer needs no "read" barrier: block i + 2 is staged into the buffer
    // of block i - 2 only after the MMAs of block i - 2 completed, and those
    // waited for every producer's fill of that block.
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_in + kMmaStaging * kMmaStageInPad);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(s_bar + 10);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_bar + 11);
    volatile int* s_issued = reinterpret_cast<volatile int*>(s_bar + 12);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c_begin = static_cast<int64_t>(blockIdx.x) * A.spins_per_cta;
    const int64_t c_end = min(A.n, c_begin + A.spins_per_cta);
    const int n_chunks = c_end > c_begin ? static_cast<int>((c_end - c_begin + kMmaChunk - 1) / kMmaChunk) : 0;
    const int n_it = n_chunks * A.n_groups;
    const uint32_t bar0 = smem_u32(s_bar);
    auto full = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(i); };
    auto empty = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(2 + i); };
    auto acc_free = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(4 + i); };
    auto staged = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(6 + i); };
    constexpr int kEWarps = kMmaThreads / 32;
    constexpr int kMmaWarp = (kMmaThreads + kMmaZThreads) / 32;

    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                     "r"(kMmaTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(full(i), kMmaThreads + kMmaZThreads);
            mbar_init(empty(i), 1);
            mbar_init(acc_free(i), kMmaThreads);
        }
        for (int i = 0; i < kMmaStaging; ++i) mbar_init(staged(i), kMmaThreads);
        *s_abort = 0;
        *s_issued = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_taddr;

    if (warp == kMmaWarp) {
        // ---- MMA issuer: block it into accumulator buffer (its segment) & 1
        int ch = 0, sg = 0;
        for (int it = 0; it < n_it; ++it) {
            const int st = it & 1;
            const bool seg_first = ch % kMmaSegBlocks == 0;
            bool w = true;
            if (seg_first && sg >= 2) w = mbar_wait_bounded(acc_free(sg & 1), ((sg - 2) >> 1) & 1);
            if (w) w = mbar_wait_bounded(full(st), (it >> 1) & 1);
            if (!__all_sync(kFull, w && !*s_abort)) {
                if (lane == 0) *s_abort = 1;
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t base = smem_u32(s_mma + st * kMmaStageBytes);
                const uint32_t d = tmem + static_cast<uint32_t>((sg & 1) * 128);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t ah = mma_smem_desc(base + ks * kMmaTileBytes);
                    const uint64_t al = mma_smem_desc(base + (4 + ks) * kMmaTileBytes);
                    const uint64_t bh = mma_smem_desc(base + (8 + ks) * kMmaTileBytes);
                    const uint64_t bl = mma_smem_desc(base + (12 + ks) * kMmaTileBytes);
                    tc_mma_f16(d, ah, bh, (!seg_first || ks > 0) ? 1u : 0u);
                    tc_mma_f16(d, ah, bl, 1u);
                    tc_mma_f16(d, al, bh, 1u);
                }
                tc_commit(empty(st));
                *s_issued = it + 1;
            }
            __syncwarp();
            if ((ch + 1) % kMmaSegBlocks == 0 || ch + 1 == n_chunks) ++sg;
            if (++ch == n_chunks) ch = 0;
        }
    } else if (warp >= kEWarps) {
        // ---- B-slice producers: the rotator powers of each block once its
        // stage is free and its staging has landed
        const int v = warp - kEWarps;
        int gi = 0, ch = 0;
        MmaGroupPk gpk;
        if (n_it > 0) gpk.set(A.groups[0]);
        for (int it = 0; it < n_it; ++it) {
            const int st = it & 1, buf = it % kMmaStaging;
            bool w = true;
            if (it >= 2) w = mbar_wait_bounded(empty(st), ((it - 2) >> 1) & 1);
            if (w) w = mbar_wait_bounded(staged(buf), (it / kMmaStaging) & 1);
            if (!w || *s_abort) {
                *s_abort = 1;
                break;
            }
            mma_fill_z(s_mma + st * kMmaStageBytes, s_in + buf * kMmaStageInPad, gpk, v, lane);
            fence_proxy_async_smem();
            mbar_arrive(full(st));
            if (++ch == n_chunks) {
                ch = 0;
                if (++gi < A.n_groups) gpk.set(A.groups[gi]);
            }
        }
    } else {
        // ---- E-slice producers: staging two blocks ahead, the A slices from
        // the staging, each group's epilogue
        float* __restrict__ out = reinterpret_cast<float*>(A.partial + static_cast<int64_t>(blockIdx.x) * A.n_adc);
        MmaStager pf;
        int pg = 0, pc = 0;  // (group, block) of the next block to stage
        auto stage_next = [&](int k) {
            pf.stage(smem_u32(s_in + (k % kMmaStaging) * kMmaStageInPad), A, pg,
                     c_begin + static_cast<int64_t>(pc) * kMmaChunk, tid);
            cp_async_arrive(staged(k % kMmaStaging));
            if (++pc == n_chunks) {
                pc = 0;
                ++pg;
            }
        };
        for (int k = 0; k < 2 && k < n_it; ++k) stage_next(k);
        int gi = 0, ch = 0, sg = 0;
        MmaGroup G = n_it > 0 ? A.groups[0] : MmaGroup{};
        // this thread's run of the E slices (run 4 warp + lane % 4 of the group)
        const int my_r = 4 * warp + (lane & 3);
        MmaRunPk my_run;
        if (n_it > 0 && my_r < G.n_runs) my_run.set(A.runs[G.run0 + my_r]);
        for (int it = 0; it < n_it; ++it) {
            const int st = it & 1, buf = it % kMmaStaging;
            bool w = true;
            if (it >= 2) w = mbar_wait_bounded(empty(st), ((it - 2) >> 1) & 1);  // MMAs of block it - 2 done
            // staging buffer (it + 2) % 4 last held block it - 2, read before
            // those MMAs were issued
            if (w && it + 2 < n_it) stage_next(it + 2);
            if (w) w = mbar_wait_bounded(staged(buf), (it / kMmaStaging) & 1);
            if (!w || *s_abort) {
                *s_abort = 1;
                break;
            }
            const int64_t s0 = c_begin + static_cast<int64_t>(ch) * kMmaChunk;
            const int live = static_cast<int>(min(static_cast<int64_t>(kMmaChunk), c_end - s0));
            unsigned char* stage = s_mma + st * kMmaStageBytes;
            const unsigned char* in = s_in + buf * kMmaStageInPad;
            mma_fill_e<kZ, kDF>(stage, in, my_run, my_r < G.n_runs, G.one_snap != 0, live, warp, lane);
            fence_proxy_async_smem();
            mbar_arrive(full(st));
            const bool grp_last = ch + 1 == n_chunks;
            if ((ch + 1) % kMmaSegBlocks != 0 && !grp_last) {
                ++ch;
                continue;
            }
            // drain of the segment: its last commit covers all its MMAs
            if (!mbar_wait_bounded(empty(st), (it >> 1) & 1) || *s_abort) {
                *s_abort = 1;
                break;
            }
            tc_fence_after();
            const bool grp_first = ch < kMmaSegBlocks;
            const int quarter = warp & 3, cgrp = warp >> 2;
            const int row = 32 * quarter + lane, r = row >> 1, part = row & 1;
            const uint32_t lanes = static_cast<uint32_t>(32 * quarter) << 16;
            int64_t run_k0 = 0;
            int run_len = 0;
            if (grp_last && r < G.n_runs) {
                run_k0 = A.runs[G.run0 + r].k0;
                run_len = A.runs[G.run0 + r].len;
                if (run_k0 < 0 || run_k0 + run_len > A.n_adc || run_len > kMaxAdcRun) {  // 128 accumulator columns
                    atomicOr(A.status, kStatusBadRun);
                    run_len = 0;
                }
            }
#pragma unroll 1
            for (int cc = 0; cc < 32; cc += 4) {
                const uint32_t col0 = static_cast<uint32_t>(32 * cgrp + cc);
                uint32_t rv[4], rs[4];
                tc_ld4(tmem + lanes + static_cast<uint32_t>((sg & 1) * 128) + col0, rv);
                if (!grp_first) tc_ld4(tmem + lanes + kMmaSumCol + col0, rs);
                tc_wait_ld();
                float v[4], sm[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x = __uint_as_float(rv[q]);
                    if (grp_first) {
                        // the group's first segment: sum = x, error = 0
                        sm[q] = x;
                        v[q] = 0.f;
                    } else {
                        // TwoSum: sum + x = t + e exactly; v <- e
                        const float a = __uint_as_float(rs[q]);
                        const float t = a + x;
                        const float z = t - a;
                        v[q] = (a - (t - z)) + (x - z);
                        sm[q] = t;
                    }
                }
                if (!grp_first) {
                    // plus the errors of the earlier segments
                    tc_ld4(tmem + lanes + kMmaErrCol + col0, rs);
                    tc_wait_ld();
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] += __uint_as_float(rs[q]);
                }
                if (grp_last) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = static_cast<int>(col0) + q;
                        if (c < run_len) out[2 * (run_k0 + c) + part] = (sm[q] + v[q]) * A.einv;
                    }
                } else {
                    tc_st4(tmem + lanes + kMmaSumCol + col0, sm);
                    tc_st4(tmem + lanes + kMmaErrCol + col0, v);
                }
            }
            if (!grp_last) tc_wait_st();
            tc_fence_before();
            mbar_arrive(acc_free(sg & 1));
            ++sg;
            if (!grp_last) {
                ++ch;
                continue;
            }
            ch = 0;
            if (++gi < A.n_groups) {
                G = A.groups[gi];
                if (my_r < G.n_runs) my_run.set(A.runs[G.run0 + my_r]);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    if (*s_abort && tid == 0) {
        atomicOr(A.status, kStatusTimeout);
        // tensor memory is released only after every issued MMA completed
        // (commits complete in order: wait for the latest)
        const int n = *s_issued;
        if (n > 0) mbar_wait_bounded(empty((n - 1) & 1), ((n - 1) >> 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmaTmemCols)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Phantom conversion (upload): the FP32 block from the FP64 rows, element by
// element. hi = float(v), lo = float(v - hi), log2(e)/T in FP64 then rounded
// (T = +inf gives 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_f64(double v, float* hi, float* lo) {
    const float h = __double2float_rn(v);
    *hi = h;
    *lo = __double2float_rn(v - static_cast<double>(h));
}

__global__ void __launch_bounds__(256) phantom_convert_kernel(double* __restrict__ p64, float* __restrict__ p32,
                                                              int64_t n, int64_t np, ConvertStatus* __restrict__ cs) {
    const double kLog2e = 1.44269504088896340736;
    double ext[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < np;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (j < n) {
            const double x = p64[P64_X * np + j], y = p64[P64_Y * np + j], z = p64[P64_Z * np + j];
            const double dw = p64[P64_F * np + j], t1 = p64[P64_T1 * np + j], t2 = p64[P64_T2 * np + j];
            const double pd = p64[P64_M0 * np + j];
            // the upload's input checks: finite x, y, z, dw and pd >= 0; T1, T2 > 0 (+inf allowed)
            const bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(dw) && isfinite(pd) && pd >= 0.0 &&
                            t1 > 0.0 && !isnan(t1) && t2 > 0.0 && !isnan(t2);
            if (!ok) atomicMin(&cs->first_bad, static_cast<unsigned long long>(j));
            const double f = dw / (2.0 * 3.14159265358979323846);
            split_f64(x, &p32[P32_XH * np + j], &p32[P32_XL * np + j]);
            split_f64(y, &p32[P32_YH * np + j], &p32[P32_YL * np + j]);
            split_f64(z, &p32[P32_ZH * np + j], &p32[P32_ZL * np + j]);
            split_f64(f, &p32[P32_FH * np + j], &p32[P32_FL * np + j]);
            p32[P32_M0 * np + j] = __double2float_rn(pd);
            p32[P32_R1 * np + j] = __double2float_rn(kLog2e / t1);
            p32[P32_R2 * np + j] = __double2float_rn(kLog2e / t2);
            p64[P64_F * np + j] = f;
            if (ok) {
                ext[0] = fmax(ext[0], fabs(x));
                ext[1] = fmax(ext[1], fabs(y));
                ext[2] = fmax(ext[2], fabs(z));
                ext[3] = fmax(ext[3], fabs(dw) / (2.0 * 3.14159265358979323846));
                ext[4] = fmax(ext[4], pd);
            }
        } else {
            for (int r = 0; r < P32_N; ++r) p32[r * np + j] = 0.f;
            for (int r = 0; r < P64_N; ++r) p64[r * np + j] = (r == P64_T1 || r == P64_T2) ? 1.0 : 0.0;
        }
    }
    // extents: warp maxima, then one atomic per warp on the bit patterns
    // (non-negative doubles order like their bits as unsigned integers)
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        double v = ext[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
        if ((threadIdx.x & 31) == 0 && v > 0.0)
            atomicMax(&cs->max_bits[d], static_cast<unsigned long long>(__double_as_longlong(v)));
    }
}

// ---------------------------------------------------------------------------
// Self-check of the device-side timeout path: one thread waits, with the
// bounded wait the Bloch kernels use on their record tiles, on an mbarrier
// that nothing completes (no copy is ever issued to it). After `limit_ns` it
// gives up, sets bit 1 of the status word and returns; the next koma_sync
// reports KOMA_E_TIMEOUT and the context stays usable.
// ---------------------------------------------------------------------------
__global__ void bounded_wait_check_kernel(int* status, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t s_bar;
    const uint32_t bar = smem_u32(&s_bar);
    mbar_init(bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(bar, 0, limit_ns)) atomicOr(status, kStatusWaitCheck);
}

// ---------------------------------------------------------------------------
// K2: sig[g][k] = sum over the CTAs c of group g of partial[c][k] in a fixed
// order (deterministic; threadIdx.y strides the CTAs, the eight strided sums
// are then added in y order in FP64). FP32 rows are summed with an error-free
// transformation per addition (Knuth's TwoSum: s + x = t + e exactly, t the
// rounded sum), the errors e collected in a second FP32 accumulator and the
// two joined in FP64: the result is the exact sum up to that accumulator's
// own rounding, about n 2^-48 of the sum of magnitudes for n rows — as close
// as FP64 additions — at FP32 speed: the part's FP64 unit runs at 1/64 of
// the FP32 rate, and plain FP64 additions bounded this kernel (epi512 0.029
// -> 0.010 ms). FP64 rows are added in FP64.
// ---------------------------------------------------------------------------

// rows c_lo, c_lo + c_step, ... < c_hi of column k, in that order
__device__ __forceinline__ void strided_sum(const float2* __restrict__ part, int64_t n_adc, int64_t k, int c_lo,
                                            int c_hi, int c_step, double& re, double& im) {
    TwoSumAcc a, b;
#pragma unroll 4
    for (int c = c_lo; c < c_hi; c += c_step) {
        const float2 p = part[static_cast<int64_t>(c) * n_adc + k];
        a.add(p.x);
        b.add(p.y);
    }
    re = a.value();
    im = b.value();
}
__device__ __forceinline__ void strided_sum(const double2* __restrict__ part, int64_t n_adc, int64_t k, int c_lo,
                                            int c_hi, int c_step, double& re, double& im) {
    double x = 0.0, y = 0.0;
#pragma unroll 4
    for (int c = c_lo; c < c_hi; c += c_step) {
        const double2 p = part[static_cast<int64_t>(c) * n_adc + k];
        x += p.x;
        y += p.y;
    }
    re = x;
    im = y;
}

template <typename P>
__global__ void __launch_bounds__(256) reduce_partials_kernel(const __grid_constant__ ReduceArgs R) {
    __shared__ double s_re[8][32];
    __shared__ double s_im[8][32];
    const int64_t chunks = (R.n_adc + 31) / 32;
    const int64_t g = blockIdx.x / chunks;
    const int64_t k = (blockIdx.x % chunks) * 32 + threadIdx.x;
    // samples of the matrix-form readout sum its rows instead (one group)
    const bool mm = R.from_mma != nullptr && k < R.n_adc && R.from_mma[k] != 0;
    const int c_lo = mm ? 0 : (R.group_cta ? R.group_cta[g] : 0);
    const int c_hi = mm ? R.grid_mma : (R.group_cta ? R.group_cta[g + 1] : R.grid);
    const P* __restrict__ part = static_cast<const P*>(mm ? R.partial_mma : R.partial);
    double re = 0.0, im = 0.0;
    if (k < R.n_adc) strided_sum(part, R.n_adc, k, c_lo + static_cast<int>(threadIdx.y), c_hi, 8, re, im);
    s_re[threadIdx.y][threadIdx.x] = re;
    s_im[threadIdx.y][threadIdx.x] = im;
    __syncthreads();
    if (threadIdx.y == 0 && k < R.n_adc) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            a += s_re[y][threadIdx.x];
            b += s_im[y][threadIdx.x];
        }
        R.sig[2 * (g * R.n_adc + k)] = a;
        R.sig[2 * (g * R.n_adc + k) + 1] = b;
    }
}

// The same sum for launches whose groups hold few rows each (the grouped
// work-item kernel: a few items per dictionary entry): one thread per
// (group, sample) adds the group's rows in order (deterministic), so a block
// covers 256 samples of one group instead of 32 samples with mostly idle
// row lanes.
template <typename P>
__global__ void __launch_bounds__(256) reduce_rows_kernel(const __grid_constant__ ReduceArgs R) {
    const int64_t chunks = (R.n_adc + 255) / 256;
    const int64_t g = blockIdx.x / chunks;
    const int64_t k = (blockIdx.x % chunks) * 256 + threadIdx.x;
    if (k >= R.n_adc) return;
    const int c_lo = R.group_cta ? R.group_cta[g] : 0;
    const int c_hi = R.group_cta ? R.group_cta[g + 1] : R.grid;
    const P* __restrict__ part = static_cast<const P*>(R.partial);
    double re = 0.0, im = 0.0;
    strided_sum(part, R.n_adc, k, c_lo, c_hi, 1, re, im);
    R.sig[2 * (g * R.n_adc + k)] = re;
    R.sig[2 * (g * R.n_adc + k) + 1] = im;
}

size_t fp32_dyn_smem(int block) { return static_cast<size_t>(2 * (block / 32) * kRed32) * sizeof(float2); }

template <int S>
cudaError_t prepare_fp32(size_t dyn) {
    cudaError_t e = cudaFuncSetAttribute(bloch_fp32_kernel<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(bloch_fp32_kernel<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(dyn));
}

template <int S>
cudaError_t occupancy_fp32(int* n, int block, size_t dyn) {
    cudaError_t e = prepare_fp32<S>(fp32_dyn_smem(kMaxBlock));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, bloch_fp32_kernel<S, false>, block, dyn);
}

template <int S>
cudaError_t launch_fp32(const BlochArgs& a, const BlochLaunch& L, cudaStream_t st) {
    const size_t dyn = fp32_dyn_smem(L.block);
    // the kernel's dynamic shared-memory limit is process-wide: set it to what
    // the largest block needs (never lower), so launches from other threads
    // with larger blocks are not invalidated between their set-up and launch
    cudaError_t e = prepare_fp32<S>(fp32_dyn_smem(kMaxBlock));
    if (e != cudaSuccess) return e;
    if (a.split > 1)
        bloch_fp32_kernel<S, true><<<L.grid, L.block, dyn, st>>>(a);
    else
        bloch_fp32_kernel<S, false><<<L.grid, L.block, dyn, st>>>(a);
    return cudaGetLastError();
}

cudaError_t prepare_motion(size_t dyn) {
    cudaError_t e = cudaFuncSetAttribute(bloch_motion_kernel<kMotionSpinsPerThread, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(bloch_motion_kernel<kMotionSpinsPerThread, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
}

template <int S, int T>
cudaError_t occupancy_items(int* n, int block) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, bloch_items_kernel<S, T, false>, block, 0);
}

}  // namespace

int bloch_max_block() { return kMaxBlock; }

int items_ctas_per_sm(int spins_per_thread, int block, int tile) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (spins_per_thread == 2)
        e = tile == 256 ? occupancy_items<2, 256>(&n, block)
                        : tile == 128 ? occupancy_items<2, 128>(&n, block) : occupancy_items<2, 64>(&n, block);
    else if (spins_per_thread == 4)
        e = tile == 256 ? occupancy_items<4, 256>(&n, block)
                        : tile == 128 ? occupancy_items<4, 128>(&n, block) : occupancy_items<4, 64>(&n, block);
    return e == cudaSuccess ? n : -1;
}

int batches_ctas_per_sm(int block) {
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_batches_kernel<4>, block, 0) == cudaSuccess ? n
                                                                                                            : -1;
}

int launch_batches(const BatchArgs& a, int grid, int block, void* stream) {
    if (block <= 0 || block > kMaxBlock || block % 32 != 0 || grid <= 0) return cudaErrorInvalidValue;
    bloch_batches_kernel<4><<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError();
}

int launch_items_z(const ItemArgs& a, int grid, int block, int tile, bool small_phase, void* stream) {
    if (block <= 0 || block > (small_phase ? kZSmallBlock : kMaxBlock) || block % 32 != 0 || grid <= 0)
        return cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (tile == 128 && small_phase) bloch_items_z_kernel<128, true><<<grid, block, 0, st>>>(a);
    else if (tile == 128) bloch_items_z_kernel<128, false><<<grid, block, 0, st>>>(a);
    else if (tile == 256 && small_phase) bloch_items_z_kernel<256, true><<<grid, block, 0, st>>>(a);
    else if (tile == 256) bloch_items_z_kernel<256, false><<<grid, block, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int items_z_ctas_per_sm(int block, int tile, bool small_phase) {
    int n = 0;
    cudaError_t e;
    if (tile == 256)
        e = small_phase ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_items_z_kernel<256, true>, block, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_items_z_kernel<256, false>, block, 0);
    else
        e = small_phase ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_items_z_kernel<128, true>, block, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_items_z_kernel<128, false>, block, 0);
    return e == cudaSuccess ? n : -1;
}

int launch_items(const ItemArgs& a, int grid, int block, int spins_per_thread, int tile, void* stream) {
    if (block <= 0 || block > kMaxBlock || block % 32 != 0 || grid <= 0) return cudaErrorInvalidValue;
    if (tile != 64 && tile != 128 && tile != 256) return cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int key = (a.uni_relax ? 10000 : 0) + spins_per_thread * 1000 + tile;
    switch (key) {
        case 2064: bloch_items_kernel<2, 64, false><<<grid, block, 0, st>>>(a); break;
        case 2128: bloch_items_kernel<2, 128, false><<<grid, block, 0, st>>>(a); break;
        case 2256: bloch_items_kernel<2, 256, false><<<grid, block, 0, st>>>(a); break;
        case 4064: bloch_items_kernel<4, 64, false><<<grid, block, 0, st>>>(a); break;
        case 4128: bloch_items_kernel<4, 128, false><<<grid, block, 0, st>>>(a); break;
        case 4256: bloch_items_kernel<4, 256, false><<<grid, block, 0, st>>>(a); break;
        case 12064: bloch_items_kernel<2, 64, true><<<grid, block, 0, st>>>(a); break;
        case 12128: bloch_items_kernel<2, 128, true><<<grid, block, 0, st>>>(a); break;
        case 12256: bloch_items_kernel<2, 256, true><<<grid, block, 0, st>>>(a); break;
        case 14064: bloch_items_kernel<4, 64, true><<<grid, block, 0, st>>>(a); break;
        case 14128: bloch_items_kernel<4, 128, true><<<grid, block, 0, st>>>(a); break;
        case 14256: bloch_items_kernel<4, 256, true><<<grid, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int bloch_ctas_per_sm(bool fp64, int spins_per_thread, int block) {
    int n = 0;
    cudaError_t e;
    if (fp64) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_fp64_kernel<false>, block, 0);
    } else {
        const size_t dyn = fp32_dyn_smem(block);
        switch (spins_per_thread) {
            case 2: e = occupancy_fp32<2>(&n, block, dyn); break;
            case 4: e = occupancy_fp32<4>(&n, block, dyn); break;
            default: return -1;
        }
    }
    return e == cudaSuccess ? n : -1;
}

int launch_bloch_fp32(const BlochArgs& a, const BlochLaunch& L, void* stream) {
    if (L.block <= 0 || L.block > kMaxBlock || L.block % 32 != 0 || L.grid <= 0) return cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (L.spins_per_thread) {
        case 2: return launch_fp32<2>(a, L, st);
        case 4: return launch_fp32<4>(a, L, st);
        default: return cudaErrorInvalidValue;
    }
}

size_t motion_dyn_smem(int block) {
    return fp32_dyn_smem(block) + static_cast<size_t>(7 * kMotionSpinsPerThread * block) * sizeof(float);
}

int motion_ctas_per_sm(int block) {
    const size_t dyn = motion_dyn_smem(block);
    if (prepare_motion(motion_dyn_smem(kMaxBlock)) != cudaSuccess) return -1;
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bloch_motion_kernel<kMotionSpinsPerThread, false>,
                                                         block, dyn) == cudaSuccess ? n : -1;
}

int launch_bloch_motion(const BlochArgs& a, const BlochLaunch& L, void* stream) {
    if (L.block <= 0 || L.block > kMaxBlock || L.block % 32 != 0 || L.grid <= 0 ||
        L.spins_per_thread != kMotionSpinsPerThread || !a.pv32)
        return cudaErrorInvalidValue;
    const size_t dyn = motion_dyn_smem(L.block);
    cudaError_t e = prepare_motion(motion_dyn_smem(kMaxBlock));  // never lowered (see launch_fp32)
    if (e != cudaSuccess) return e;
    if (a.split > 1)
        bloch_motion_kernel<kMotionSpinsPerThread, true><<<L.grid, L.block, dyn, static_cast<cudaStream_t>(stream)>>>(a);
    else
        bloch_motion_kernel<kMotionSpinsPerThread, false><<<L.grid, L.block, dyn, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError();
}

int launch_rf_maps(const RfMapArgs& a, void* stream) {
    if (a.n_pulses <= 0 || a.n_pulses > kMaxRfMaps || a.n <= 0) return cudaErrorInvalidValue;
    const int64_t gx = (a.n + 2 * kMapBlock - 1) / (2 * kMapBlock);
    if (gx > 0x7fffffff) return cudaErrorInvalidValue;
    rf_map_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(a.n_pulses)), kMapBlock, 0,
                    static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError();
}

int launch_bloch_fp64(const BlochArgs& a, const BlochLaunch& L, void* stream) {
    if (L.block <= 0 || L.block > kMaxBlock || L.block % 32 != 0 || L.grid <= 0 || L.spins_per_thread != 1)
        return cudaErrorInvalidValue;
    bloch_fp64_kernel<false><<<L.grid, L.block, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError();
}

int launch_bloch_fp64_motion(const BlochArgs& a, const BlochLaunch& L, void* stream) {
    if (L.block <= 0 || L.block > kMaxBlock || L.block % 32 != 0 || L.grid <= 0 || L.spins_per_thread != 1 ||
        !a.pv64)
        return cudaErrorInvalidValue;
    bloch_fp64_kernel<true><<<L.grid, L.block, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Static scratch for koma_simulate_static (callers that cannot allocate
// device memory). A file-scope device array of kStaticPartials float2
// (32 MiB) that every GPU loading this library holds until exit. In host
// code `g_static_partials` is only a host-side stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress, taken once per device
// (with that device current) and cached. All calls share the array.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kStaticPartials = size_t(4) << 20;  // float2 elements = 32 MiB
constexpr int kMaxDevices = 64;
static __device__ __align__(256) float2 g_static_partials[kStaticPartials];
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
}  // namespace

size_t static_partials_capacity() { return kStaticPartials; }

int static_partials_ptr(int device, void** out) {
    *out = nullptr;
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[device]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != device) return cudaErrorInvalidDevice;  // caller makes `device` current
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return e;
        g_static_ptr[device] = p;
    }
    *out = g_static_ptr[device];
    return cudaSuccess;
}

int launch_phantom_convert(double* p64, float* p32, int64_t n, int64_t n_pad, ConvertStatus* cs, void* stream) {
    if (n_pad <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n_pad + 255) / 256, 148 * 16);
    phantom_convert_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(p64, p32, n,
                                                                                                         n_pad, cs);
    return cudaGetLastError();
}

int launch_bounded_wait_check(int* status, unsigned long long limit_ns, void* stream) {
    bounded_wait_check_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(status, limit_ns);
    return cudaGetLastError();
}

template <bool kZ, bool kDF>
static int launch_readout_mma_t(const MmaArgs& a, int grid, cudaStream_t st) {
    const cudaError_t attr = cudaFuncSetAttribute(readout_mma_kernel<kZ, kDF>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  static_cast<int>(kMmaDynSmem));
    if (attr != cudaSuccess) return attr;
    readout_mma_kernel<kZ, kDF><<<static_cast<unsigned>(grid), kMmaCtaThreads, kMmaDynSmem, st>>>(a);
    return cudaGetLastError();
}

int launch_readout_mma(const MmaArgs& a, int grid, void* stream) {
    if (grid <= 0 || a.spins_per_cta % kMmaChunk != 0 || a.n_pad % 2 != 0) return cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool z = (a.used & 4) != 0, df = (a.used & 8) != 0;
    if (z) return df ? launch_readout_mma_t<true, true>(a, grid, st) : launch_readout_mma_t<true, false>(a, grid, st);
    return df ? launch_readout_mma_t<false, true>(a, grid, st) : launch_readout_mma_t<false, false>(a, grid, st);
}

int launch_reduce(const ReduceArgs& r, bool fp64_partials, void* stream) {
    if (r.n_adc <= 0 || r.n_groups <= 0) return cudaSuccess;
    if (r.from_mma == nullptr && r.grid <= 8 * r.n_groups) {
        // few rows a group (<= 8 on average)
        const int64_t blocks = (r.n_adc + 255) / 256 * r.n_groups;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (fp64_partials)
            reduce_rows_kernel<double2><<<static_cast<unsigned>(blocks), 256, 0, st>>>(r);
        else
            reduce_rows_kernel<float2><<<static_cast<unsigned>(blocks), 256, 0, st>>>(r);
        return cudaGetLastError();
    }
    const int64_t chunks = (r.n_adc + 31) / 32;
    const int64_t blocks = chunks * r.n_groups;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 blk(32, 8);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (fp64_partials)
        reduce_partials_kernel<double2><<<static_cast<unsigned>(blocks), blk, 0, st>>>(r);
    else
        reduce_partials_kernel<float2><<<static_cast<unsigned>(blocks), blk, 0, st>>>(r);
    return cudaGetLastError();
}

}  // namespace koma
