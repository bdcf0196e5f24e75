// Device helpers shared by the kernels of libpfb: complex arithmetic,
// in-register small DFTs, input loaders for the three sample types, stores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pfb {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// b * exp(-2 pi i m / 16) for a compile-time m in [0, 8) (after unrolling the
// switch folds away).  Constants: cos(pi/8), sin(pi/8), sqrt(1/2).
__device__ __forceinline__ float2 twmul16(float2 b, int m) {
    constexpr float C1 = 0.92387953251128674f;
    constexpr float S1 = 0.38268343236508977f;
    constexpr float H = 0.70710678118654752f;
    switch (m) {
    case 0: return b;
    case 1: return cmul(b, make_float2(C1, -S1));
    case 2: return make_float2(H * (b.x + b.y), H * (b.y - b.x));
    case 3: return cmul(b, make_float2(S1, -C1));
    case 4: return make_float2(b.y, -b.x);
    case 5: return cmul(b, make_float2(-S1, -C1));
    case 6: return make_float2(H * (b.y - b.x), -H * (b.x + b.y));
    default: return cmul(b, make_float2(-C1, -S1));
    }
}

// b * exp(-2 pi i m / 32) for a compile-time m in [0, 16)
__device__ __forceinline__ float2 twmul32(float2 b, int m) {
    if ((m & 1) == 0) return twmul16(b, m >> 1);
    switch (m) {  // cos(pi m/16), sin(pi m/16) for odd m
    case 1: return cmul(b, make_float2(0.98078528040323043f, -0.19509032201612825f));
    case 3: return cmul(b, make_float2(0.83146961230254524f, -0.55557023301960218f));
    case 5: return cmul(b, make_float2(0.55557023301960218f, -0.83146961230254524f));
    case 7: return cmul(b, make_float2(0.19509032201612825f, -0.98078528040323043f));
    case 9: return cmul(b, make_float2(-0.19509032201612825f, -0.98078528040323043f));
    case 11: return cmul(b, make_float2(-0.55557023301960218f, -0.83146961230254524f));
    case 13: return cmul(b, make_float2(-0.83146961230254524f, -0.55557023301960218f));
    default: return cmul(b, make_float2(-0.98078528040323043f, -0.19509032201612825f));
    }
}

// packed fp32x2 add / sub (Blackwell): one instruction per complex add
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\tadd.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 csub2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\tsub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// packed fp32x2 fused multiply-add: d = a * b + c on both lanes
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\tmov.b64 rc, {%6,%7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

template <int R>
__device__ __forceinline__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// One radix-2 decimation-in-time stage of butterfly span LEN over t[0..R)
// (twiddle exp(-2 pi i k / LEN) on the odd half), then the next stage.
template <int R, int LEN, bool PK>
__device__ __forceinline__ void dit_stages(float2 (&t)[R]) {
#pragma unroll
    for (int i = 0; i < R; i += LEN) {
#pragma unroll
        for (int k = 0; k < LEN / 2; ++k) {
            const float2 a = t[i + k];
            const float2 b = twmul32(t[i + k + LEN / 2], (32 / LEN) * k);
            if constexpr (PK) {
                t[i + k] = cadd2(a, b);
                t[i + k + LEN / 2] = csub2(a, b);
            } else {
                t[i + k] = cadd(a, b);
                t[i + k + LEN / 2] = csub(a, b);
            }
        }
    }
    if constexpr (LEN * 2 <= R) dit_stages<R, LEN * 2, PK>(t);
}

// In-register forward DFT, natural order in and out:
//   v[k] <- sum_r v[r] exp(-2 pi i r k / R),  R in {2, 4, 8, 16, 32}
// (iterative radix-2 decimation in time over a bit-reversed copy; PK uses
// packed fp32x2 adds for the butterflies).  Every index is a compile-time
// constant, so the arrays live in registers.
template <int R, bool PK = false>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[bitrev<R>(i)];
    dit_stages<R, 2, PK>(t);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

// ---------------------------------------------------------------------------
// input loaders: two consecutive branches (samples idx, idx+1) as complex fp32
// ---------------------------------------------------------------------------
template <int IN>
struct Loader;

template <>
struct Loader<PFB_IN_C64> {
    static constexpr bool kReal = false;
    __device__ __forceinline__ static void load2(const void *base, int64_t idx, float, float2 &a, float2 &b) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(static_cast<const float2 *>(base) + idx));
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
    }
    __device__ __forceinline__ static float2 load1(const void *base, int64_t idx, float) {
        return __ldg(static_cast<const float2 *>(base) + idx);
    }
};

template <>
struct Loader<PFB_IN_R32> {
    static constexpr bool kReal = true;
    __device__ __forceinline__ static void load2(const void *base, int64_t idx, float, float2 &a, float2 &b) {
        float2 v = __ldg(reinterpret_cast<const float2 *>(static_cast<const float *>(base) + idx));
        a = make_float2(v.x, 0.f);
        b = make_float2(v.y, 0.f);
    }
    __device__ __forceinline__ static float2 load1(const void *base, int64_t idx, float) {
        return make_float2(__ldg(static_cast<const float *>(base) + idx), 0.f);
    }
};

template <>
struct Loader<PFB_IN_CI8> {
    static constexpr bool kReal = false;
    __device__ __forceinline__ static void load2(const void *base, int64_t idx, float s, float2 &a, float2 &b) {
        char4 v = __ldg(reinterpret_cast<const char4 *>(static_cast<const int8_t *>(base) + 2 * idx));
        a = make_float2((float)v.x * s, (float)v.y * s);
        b = make_float2((float)v.z * s, (float)v.w * s);
    }
    __device__ __forceinline__ static float2 load1(const void *base, int64_t idx, float s) {
        char2 v = __ldg(reinterpret_cast<const char2 *>(static_cast<const int8_t *>(base) + 2 * idx));
        return make_float2((float)v.x * s, (float)v.y * s);
    }
};

// frame f of a stream: the state frames come first, then the input frames
__device__ __forceinline__ const void *frame_source(const StreamDesc &d, int64_t f, int64_t P, int64_t &sample) {
    if (f < d.n_state) {
        sample = f * P;
        return d.state;
    }
    sample = (f - d.n_state) * P;
    return d.in;
}

__device__ __forceinline__ void store_cs(float2 *p, float2 v) { __stcs(p, v); }

// locate the stream owning global work unit u (streams sorted by unit0)
// Report a failure code into the launch's error word (host-mapped memory: a
// plain store, made visible to the host before the kernel's completion).
__device__ __forceinline__ void report_error(int *err, int code) {
    *reinterpret_cast<volatile int *>(err) = code;
    __threadfence_system();
}

__device__ __forceinline__ int find_stream(const LaunchArgs &a, int64_t u) {
    // last stream whose first unit is <= u (unit0 ascends with the index)
    int lo = 0, hi = a.nstreams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.s[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace pfb
