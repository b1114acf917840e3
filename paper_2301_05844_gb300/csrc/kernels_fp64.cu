// FP64 / complex-FP64 kernels of the blockBP sweep and read-out.
//
// These are grouped kernels: blockIdx.y (or blockIdx.x) selects a task descriptor,
// so one launch advances every message of the sweep by one step.  They form the
// plain FP64 GPU path (every contraction, QR/LQ and reduction in FP64) and supply
// the FP64 truncation / normalisation stages of the mixed-precision path.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>

#include "bbp_internal.h"

namespace bbp {

// ---------------------------------------------------------------- scalar helpers
__device__ __forceinline__ double conjv(double a) { return a; }
__device__ __forceinline__ double2 conjv(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ void mac(double& c, double a, double b) { c = fma(a, b, c); }
__device__ __forceinline__ void mac(double2& c, double2 a, double2 b) {
    c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
}
__device__ __forceinline__ double abs2(double a) { return a * a; }
__device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
template <typename S> __device__ __forceinline__ S zero();
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ double2 zero<double2>() { return make_double2(0.0, 0.0); }
template <typename S> __device__ __forceinline__ S one();
template <> __device__ __forceinline__ double one<double>() { return 1.0; }
template <> __device__ __forceinline__ double2 one<double2>() { return make_double2(1.0, 0.0); }
template <typename S> __device__ __forceinline__ S from_real(double x);
template <> __device__ __forceinline__ double from_real<double>(double x) { return x; }
template <> __device__ __forceinline__ double2 from_real<double2>(double x) { return make_double2(x, 0.0); }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double scal(double a, double s) { return a * s; }
__device__ __forceinline__ double2 scal(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double divr(double a, double d) { return a / d; }
__device__ __forceinline__ double2 divr(double2 a, double d) { return make_double2(a.x / d, a.y / d); }
__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ double absv(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 shfl_down(double2 v, int o) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double shfl_idx(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ double2 shfl_idx(double2 v, int l) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
}
// FP32 / complex-FP32 counterparts of the helpers above (the FP32-arithmetic QR of the
// reduced-precision paths)
__device__ __forceinline__ float conjv(float a) { return a; }
__device__ __forceinline__ float2 conjv(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ void mac(float& c, float a, float b) { c = fmaf(a, b, c); }
__device__ __forceinline__ void mac(float2& c, float2 a, float2 b) {
    c.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
    c.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
}
__device__ __forceinline__ float abs2(float a) { return a * a; }
__device__ __forceinline__ float abs2(float2 a) { return a.x * a.x + a.y * a.y; }
template <> __device__ __forceinline__ float zero<float>() { return 0.0f; }
template <> __device__ __forceinline__ float2 zero<float2>() { return make_float2(0.0f, 0.0f); }
template <> __device__ __forceinline__ float one<float>() { return 1.0f; }
template <> __device__ __forceinline__ float2 one<float2>() { return make_float2(1.0f, 0.0f); }
template <> __device__ __forceinline__ float from_real<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ float2 from_real<float2>(double x) { return make_float2((float)x, 0.0f); }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float scal(float a, float s) { return a * s; }
__device__ __forceinline__ float2 scal(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float divr(float a, float d) { return a / d; }
__device__ __forceinline__ float2 divr(float2 a, float d) { return make_float2(a.x / d, a.y / d); }
__device__ __forceinline__ float absv(float a) { return fabsf(a); }
__device__ __forceinline__ float absv(float2 a) { return hypotf(a.x, a.y); }
__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shfl_down(float2 v, int o) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float shfl_idx(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float2 shfl_idx(float2 v, int l) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
}
template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
    for (int o = 16; o > 0; o >>= 1) v = add(v, shfl_down(v, o));
    return shfl_idx(v, 0);
}
// Block-wide sum for 256 threads; every thread gets the result.
template <typename S>
__device__ S block_sum(S v, S* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    S t = zero<S>();
    if (threadIdx.x < 32) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : zero<S>();
        t = warp_sum(t);
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

// Block-wide maximum for 256 threads; every thread gets the result.
__device__ double block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

__device__ float block_max(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x < 32) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_down_sync(0xffffffffu, t, o));
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}
// Real type of a scalar type, its FP64 counterpart, and the thresholds of the Householder
// step: a squared norm below tiny2 is recomputed relative to the largest entry (its squares
// would lose bits to underflow), and a divisor below tiny_div is divided by instead of
// multiplied by its reciprocal (which would overflow).
template <typename S> struct ScalarTraits;
template <> struct ScalarTraits<double> {
    using R = double;
    using Wide = double;
    static __device__ __forceinline__ double tiny2() { return 1e-280; }
    static __device__ __forceinline__ double tiny_div() { return 1e-290; }
};
template <> struct ScalarTraits<double2> {
    using R = double;
    using Wide = double2;
    static __device__ __forceinline__ double tiny2() { return 1e-280; }
    static __device__ __forceinline__ double tiny_div() { return 1e-290; }
};
template <> struct ScalarTraits<float> {
    using R = float;
    using Wide = double;
    static __device__ __forceinline__ float tiny2() { return 1e-30f; }
    static __device__ __forceinline__ float tiny_div() { return 1e-36f; }
};
template <> struct ScalarTraits<float2> {
    using R = float;
    using Wide = double2;
    static __device__ __forceinline__ float tiny2() { return 1e-30f; }
    static __device__ __forceinline__ float tiny_div() { return 1e-36f; }
};
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double hypot_r(double a, double b) { return hypot(a, b); }
__device__ __forceinline__ double max_r(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float max_r(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float max_component(float a) { return fabsf(a); }
__device__ __forceinline__ float max_component(float2 a) { return fmaxf(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float hypot_r(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double widen(double a) { return a; }
__device__ __forceinline__ double2 widen(double2 a) { return a; }
__device__ __forceinline__ double widen(float a) { return (double)a; }
__device__ __forceinline__ double2 widen(float2 a) { return make_double2((double)a.x, (double)a.y); }
// (h, l) <- h + c exactly as the pair h + l (Knuth's TwoSum; l collects the rounding errors)
__device__ __forceinline__ void two_sum_into(float& h, float& l, float c) {
    const float s = h + c, bp = s - h;
    l += (h - (s - bp)) + (c - bp);
    h = s;
}
__device__ __forceinline__ void two_sum_into(float2& h, float2& l, float2 c) {
    two_sum_into(h.x, l.x, c.x);
    two_sum_into(h.y, l.y, c.y);
}
__device__ __forceinline__ void two_sum_into(double&, double&, double) {}
__device__ __forceinline__ void two_sum_into(double2&, double2&, double2) {}
template <typename Cm> __device__ __forceinline__ Cm narrow(double a);
template <typename Cm> __device__ __forceinline__ Cm narrow(double2 a);
template <> __device__ __forceinline__ double narrow<double>(double a) { return a; }
template <> __device__ __forceinline__ double2 narrow<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float narrow<float>(double a) { return (float)a; }
template <> __device__ __forceinline__ float2 narrow<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---------------------------------------------------------------- SplitMix64
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double u_pm1(uint64_t key, uint64_t idx) {
    return (double)(sm64(key + idx) >> 11) * 0x1.0p-52 - 1.0;
}
uint64_t splitmix64(uint64_t z) { return sm64(z); }
// key = splitmix64(seed XOR splitmix64(stream)); value i = splitmix64(key + i) mapped to [-1, 1)
__host__ __device__ __forceinline__ uint64_t rng_key(uint64_t seed, uint64_t stream) { return sm64(seed ^ sm64(stream)); }
double uniform_pm1(uint64_t seed, uint64_t stream, uint64_t idx) { return u_pm1(rng_key(seed, stream), idx); }

// ---------------------------------------------------------------- element kinds
template <typename S> __device__ __forceinline__ S from_float(const float* p, long long i);
template <> __device__ __forceinline__ double from_float<double>(const float* p, long long i) { return (double)p[i]; }
template <> __device__ __forceinline__ double2 from_float<double2>(const float* p, long long i) {
    return make_double2((double)p[2 * i], (double)p[2 * i + 1]);
}
template <> __device__ __forceinline__ float from_float<float>(const float* p, long long i) { return p[i]; }
template <> __device__ __forceinline__ float2 from_float<float2>(const float* p, long long i) {
    return make_float2(p[2 * i], p[2 * i + 1]);
}
// element i of an FP64 (complex-FP64) array in the scalar type S
template <typename S> __device__ __forceinline__ S from_double(const void* p, long long i);
template <> __device__ __forceinline__ double from_double<double>(const void* p, long long i) { return ((const double*)p)[i]; }
template <> __device__ __forceinline__ double2 from_double<double2>(const void* p, long long i) {
    return ((const double2*)p)[i];
}
template <> __device__ __forceinline__ float from_double<float>(const void* p, long long i) {
    return (float)((const double*)p)[i];
}
template <> __device__ __forceinline__ float2 from_double<float2>(const void* p, long long i) {
    const double2 v = ((const double2*)p)[i];
    return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// kinds: 0 FP64, 2 FP32, 3 BF16, 4 FP32 rounded to TF32
__device__ __forceinline__ void store_kind(void* p, long long i, int kind, double v) {
    switch (kind) {
        case 0: ((double*)p)[i] = v; break;
        case 2: ((float*)p)[i] = (float)v; break;
        case 3: ((__nv_bfloat16*)p)[i] = __double2bfloat16(v); break;
        default: ((float*)p)[i] = tf32_round((float)v); break;
    }
}
__device__ __forceinline__ void store_kind(void* p, long long i, int kind, double2 v) {
    store_kind(p, 2 * i, kind, v.x);
    store_kind(p, 2 * i + 1, kind, v.y);
}
// Split operand (x3 != 0; kind 4 TF32, kind 3 BF16): hi = r(v), lo = r(v - hi), r the rounding
// of the kind applied to the FP32 rounding of v; hi goes to the first plane, lo kseg elements
// further (the second plane).  A consumer GEMM reads them as the K-segments (hi, lo, hi) of an A
// operand or (hi, hi, lo) of a B operand, forming A_hi B_hi + A_lo B_hi + A_hi B_lo.
__device__ __forceinline__ void store_split(void* p, long long i, int kind, double v, int x3, long long kseg) {
    if (!x3) {
        store_kind(p, i, kind, v);
        return;
    }
    const float f32 = (float)v;
    if (kind == 3) {
        const __nv_bfloat16 hb = __float2bfloat16_rn(f32);
        const __nv_bfloat16 lb = __float2bfloat16_rn(f32 - __bfloat162float(hb));  // f32 - hi is exact
        __nv_bfloat16* b = (__nv_bfloat16*)p;
        b[i] = hb;
        b[i + kseg] = lb;
        return;
    }
    const float hi = tf32_round(f32), lo = tf32_round(f32 - hi);  // f32 - hi is exact
    float* f = (float*)p;
    f[i] = hi;
    f[i + kseg] = lo;
}
__device__ __forceinline__ void store_split(void* p, long long i, int kind, double2 v, int x3, long long kseg) {
    store_split(p, 2 * i, kind, v.x, x3, kseg);
    store_split(p, 2 * i + 1, kind, v.y, x3, kseg);
}
__device__ __forceinline__ double load_kind(const void* p, long long i, int kind) {
    switch (kind) {
        case 0: return ((const double*)p)[i];
        case 2: case 4: return (double)((const float*)p)[i];
        default: return (double)__bfloat162float(((const __nv_bfloat16*)p)[i]);
    }
}

// ---------------------------------------------------------------- generic contraction
// 64x64 output tile per CTA, K in chunks of 16, 256 threads each owning 4x4 outputs.
// Cm is the arithmetic type: S itself, or float / float2 for FP64 operands contracted in FP32
// arithmetic: each operand rounded to FP32 as it is staged, each chunk of 16 products summed in
// FP32 and the chunks added into an unevaluated FP32 pair (hi, lo) by Knuth's TwoSum, so that
// the accumulation error does not grow with K; the result hi + lo is formed in FP64.
template <typename S, typename Cm = S>
__global__ void __launch_bounds__(256) k_gcontract(const GTask* __restrict__ tasks) {
    const GTask& t = tasks[blockIdx.y];
    if (t.active && *t.active == 0) return;
    const int M = t.M1 * t.M2, N = t.N1 * t.N2, Kd = t.K1 * t.K2;
    const int tilesM = (M + 63) >> 6, tilesN = (N + 63) >> 6;
    const int tile = blockIdx.x;
    if (tile >= tilesM * tilesN) return;
    const int m0 = (tile % tilesM) << 6, n0 = (tile / tilesM) << 6;
    __shared__ Cm As[16][65];
    __shared__ Cm Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const S* __restrict__ Ap = (const S*)t.A;
    const S* __restrict__ Bp = (const S*)t.B;
    const int lmn = tid & 63, lk = tid >> 6;  // loader: fixed row/col, k = lk + 4j
    const int am = m0 + lmn, bn = n0 + lmn;
    const bool av = am < M, bv = bn < N;
    const long long aoff = av ? (long long)(am / t.M2) * t.a_m1 + (long long)(am % t.M2) * t.a_m2 : 0;
    const long long boff = bv ? (long long)(bn / t.N2) * t.b_n1 + (long long)(bn % t.N2) * t.b_n2 : 0;
    constexpr bool kComp = !std::is_same<S, Cm>::value;
    Cm acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = hi[i][j] = lo[i][j] = zero<Cm>();
    for (int k0 = 0; k0 < Kd; k0 += 16) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kk = lk + 4 * j, k = k0 + kk;
            S a = zero<S>(), b = zero<S>();
            if (k < Kd) {
                const int k1 = k / t.K2, k2 = k - k1 * t.K2;
                if (av) {
                    a = Ap[aoff + (long long)k1 * t.a_k1 + (long long)k2 * t.a_k2];
                    if (t.conjA) a = conjv(a);
                }
                if (bv) b = Bp[boff + (long long)k1 * t.b_k1 + (long long)k2 * t.b_k2];
            }
            As[kk][lmn] = narrow<Cm>(a);
            Bs[kk][lmn] = narrow<Cm>(b);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            Cm a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
        if constexpr (kComp) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    two_sum_into(hi[i][j], lo[i][j], acc[i][j]);
                    acc[i][j] = zero<Cm>();
                }
        }
    }
    S* __restrict__ Cp = (S*)t.C;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
        const long long mo = (long long)(m / t.M2) * t.c_m1 + (long long)(m % t.M2) * t.c_m2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            const long long o = mo + (long long)(n / t.N2) * t.c_n1 + (long long)(n % t.N2) * t.c_n2;
            S r;
            if constexpr (kComp) r = add(widen(hi[i][j]), widen(lo[i][j]));
            else r = widen(acc[i][j]);
            Cp[o] = t.accumulate ? add(Cp[o], r) : r;
        }
    }
}

// Small contractions (an output dimension of at most 16, e.g. the message overlaps): a 16x16
// output tile per CTA, one output per thread, operands read through the cache.  A 64x64 tile
// would spend most of its FP64 instructions on padding, and each warp-wide FP64 instruction
// costs the same however few lanes do useful work.  The K sum runs in four interleaved partial
// sums (four independent FP64 chains instead of one), added in a fixed order.  Cm as above.
template <typename S, typename Cm = S>
__global__ void __launch_bounds__(256) k_gcontract_small(const GTask* __restrict__ tasks) {
    const GTask& t = tasks[blockIdx.y];
    if (t.active && *t.active == 0) return;
    const int M = t.M1 * t.M2, N = t.N1 * t.N2, Kd = t.K1 * t.K2;
    const int tilesM = (M + 15) >> 4, tilesN = (N + 15) >> 4;
    if ((int)blockIdx.x >= tilesM * tilesN) return;
    const int m = ((blockIdx.x % tilesM) << 4) + (threadIdx.x & 15);
    const int n = ((blockIdx.x / tilesM) << 4) + (threadIdx.x >> 4);
    if (m >= M || n >= N) return;
    const S* __restrict__ Ap = (const S*)t.A;
    const S* __restrict__ Bp = (const S*)t.B;
    const long long aoff = (long long)(m / t.M2) * t.a_m1 + (long long)(m % t.M2) * t.a_m2;
    const long long boff = (long long)(n / t.N2) * t.b_n1 + (long long)(n % t.N2) * t.b_n2;
    Cm p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = zero<Cm>();
    int k1 = 0, k2 = 0;  // k = k1 * K2 + k2
#pragma unroll 4
    for (int k = 0; k < Kd; ++k) {
        S a = Ap[aoff + (long long)k1 * t.a_k1 + (long long)k2 * t.a_k2];
        if (t.conjA) a = conjv(a);
        mac(p[k & 3], narrow<Cm>(a), narrow<Cm>(Bp[boff + (long long)k1 * t.b_k1 + (long long)k2 * t.b_k2]));
        if (++k2 == t.K2) {
            k2 = 0;
            ++k1;
        }
    }
    const S r = widen(add(add(p[0], p[1]), add(p[2], p[3])));
    S* __restrict__ Cp = (S*)t.C;
    const long long o = (long long)(m / t.M2) * t.c_m1 + (long long)(m % t.M2) * t.c_m2 +
                        (long long)(n / t.N2) * t.c_n1 + (long long)(n % t.N2) * t.c_n2;
    Cp[o] = t.accumulate ? add(Cp[o], r) : r;
}

// FP32-arithmetic contraction of real FP64 operands with a wider tile (the read-out closings
// of tensor-core lattices): 128 x 64 outputs per CTA, K in chunks of 16, 256 threads each
// owning 8 rows x 4 columns.  The staged operands are K-major in shared memory ([k][m], [k][n])
// so that each thread reads its 8 A values and 4 B values as 16-byte vectors; the loaders walk
// m (n) fastest and keep their (k1, k2) indices incrementally (no division per element).
// Each chunk's 16 products are summed in FP32 and added into an unevaluated FP32 pair
// (hi, lo) by TwoSum, as in k_gcontract; the result hi + lo is formed in FP64.
__global__ void __launch_bounds__(256) k_gcontract_f32w(const GTask* __restrict__ tasks) {
    const GTask& t = tasks[blockIdx.y];
    if (t.active && *t.active == 0) return;
    const int M = t.M1 * t.M2, N = t.N1 * t.N2, Kd = t.K1 * t.K2;
    const int tilesM = (M + 127) >> 7, tilesN = (N + 63) >> 6;
    const int tile = blockIdx.x;
    if (tile >= tilesM * tilesN) return;
    const int m0 = (tile % tilesM) << 7, n0 = (tile / tilesM) << 6;
    __shared__ __align__(16) float As[16][128];
    __shared__ __align__(16) float Bs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const double* __restrict__ Ap = (const double*)t.A;
    const double* __restrict__ Bp = (const double*)t.B;
    // A loader: row m0 + (tid & 127), k = lk + 2j (j = 0..7); B loader: column n0 + (tid & 63), k = lkb + 4j (j = 0..3)
    const int am = m0 + (tid & 127), lk = tid >> 7;
    const int bn = n0 + (tid & 63), lkb = tid >> 6;
    const bool av = am < M, bv = bn < N;
    const long long aoff = av ? (long long)(am / t.M2) * t.a_m1 + (long long)(am % t.M2) * t.a_m2 : 0;
    const long long boff = bv ? (long long)(bn / t.N2) * t.b_n1 + (long long)(bn % t.N2) * t.b_n2 : 0;
    int ak1 = lk / t.K2, ak2 = lk - ak1 * t.K2;     // (k1, k2) of this thread's next A element
    int bk1 = lkb / t.K2, bk2 = lkb - bk1 * t.K2;  // and of its next B element
    float acc[8][4], hi[8][4], lo[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = hi[i][j] = lo[i][j] = 0.0f;
    for (int k0 = 0; k0 < Kd; k0 += 16) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int kk = lk + 2 * j;
            float a = 0.0f;
            if (av && k0 + kk < Kd) a = (float)Ap[aoff + (long long)ak1 * t.a_k1 + (long long)ak2 * t.a_k2];
            As[kk][tid & 127] = a;
            ak2 += 2;
            while (ak2 >= t.K2) {
                ak2 -= t.K2;
                ++ak1;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kk = lkb + 4 * j;
            float b = 0.0f;
            if (bv && k0 + kk < Kd) b = (float)Bp[boff + (long long)bk1 * t.b_k1 + (long long)bk2 * t.b_k2];
            Bs[kk][tid & 63] = b;
            bk2 += 4;
            while (bk2 >= t.K2) {
                bk2 -= t.K2;
                ++bk1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a0 = *(const float4*)&As[kk][ty * 8];
            const float4 a1 = *(const float4*)&As[kk][ty * 8 + 4];
            const float4 b4 = *(const float4*)&Bs[kk][tx * 4];
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                two_sum_into(hi[i][j], lo[i][j], acc[i][j]);
                acc[i][j] = 0.0f;
            }
    }
    double* __restrict__ Cp = (double*)t.C;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty * 8 + i;
        if (m >= M) continue;
        const long long mo = (long long)(m / t.M2) * t.c_m1 + (long long)(m % t.M2) * t.c_m2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            const long long o = mo + (long long)(n / t.N2) * t.c_n1 + (long long)(n % t.N2) * t.c_n2;
            const double r = (double)hi[i][j] + (double)lo[i][j];
            Cp[o] = t.accumulate ? Cp[o] + r : r;
        }
    }
}

// Layered pair contraction (GTask::layer_d > 0; read-out rows of real double-layer lattices):
// per pair, Z_p = X' Tb_p and Y' = sum_p Tk_p^T Z_p, where X' is the [(k1 k2)][(k1' k2')]
// matrix of the pair's input and Tk_p, Tb_p the [(k1 k2)][(n1 n2)] matrices of the two
// tensors: 2 d UL DR (UL + DR) flops per pair (UL = K1 K2, DR = N1 N2) where the contraction
// with the double layer E costs 2 UL^2 DR^2.  A CTA takes one m1 and APT consecutive m2 (the
// input's unit-stride index at every call site, so that the loads are contiguous runs); both
// tensors, the APT input matrices, the Z_p and the staged outputs sit in shared memory in the
// arithmetic type Cm (float: the operands are rounded to FP32 as in k_gcontract<double, float>).
// Shared layout (elements of Cm): Ts [2][d][UL][DRp] | Xs [APT][UL][ULs] (reused for the output
// tile [APT][DR*DR]) | Zs [APT][d][UL][DRp]; DRp = DR rounded up to 4 (vector reads), ULs = UL
// made odd (conflict-free row reads).
__host__ __device__ inline int layer_drp(int DR) { return (DR + 3) & ~3; }
__host__ __device__ inline int layer_uls(int UL) { return UL | 1; }
__host__ __device__ inline long long layer_round4(long long x) { return (x + 3) & ~3LL; }

__device__ inline void lds4(const float* p, float (&v)[4]) {
    const float4 q = *(const float4*)p;
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ inline void lds4(const double* p, double (&v)[4]) {
    const double2 a = *(const double2*)p, b = *(const double2*)(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename Cm, int APT>
__global__ void __launch_bounds__(256) k_layer_pair(const GTask* __restrict__ tasks) {
    const GTask& t = tasks[blockIdx.y];
    if (t.active && *t.active == 0) return;
    const int d = t.layer_d, K1 = t.K1, K2 = t.K2, N1 = t.N1, N2 = t.N2;
    const int UL = K1 * K2, DR = N1 * N2, DRp = layer_drp(DR), ULs = layer_uls(UL);
    const int tilesM2 = (t.M2 + APT - 1) / APT;
    if ((int)blockIdx.x >= t.M1 * tilesM2) return;
    const int m1 = blockIdx.x / tilesM2, m20 = (blockIdx.x % tilesM2) * APT;
    extern __shared__ __align__(16) unsigned char layer_smem[];
    Cm* Ts = (Cm*)layer_smem;
    const long long tsz = layer_round4(2LL * d * UL * DRp);
    Cm* Xs = Ts + tsz;
    const long long xin = (long long)APT * UL * ULs, xout = (long long)APT * DR * DR;
    const long long xsz = layer_round4(xin > xout ? xin : xout);
    Cm* Zs = Xs + xsz;
    const double* __restrict__ A = (const double*)t.A;
    const double* __restrict__ B = (const double*)t.B;
    const long long vol = (long long)UL * DR;
    const int tid = threadIdx.x;
    // both tensors, [side][p][(k1 k2)][(n1 n2)], pad columns zero
    for (int e = tid; e < 2 * d * UL * DRp; e += 256) {
        const int dr = e % DRp, r = e / DRp, ul = r % UL, r2 = r / UL, p = r2 % d, side = r2 / d;
        Cm v = Cm(0);
        if (dr < DR) {
            const int k1 = ul / K2, k2 = ul % K2, n1 = dr / N2, n2 = dr % N2;
            v = (Cm)B[(side ? t.tb_off : 0) + p * vol + k1 * t.b_k1 + k2 * t.b_k2 + n1 * t.b_n1 + n2 * t.b_n2];
        }
        Ts[e] = v;
    }
    // the APT input matrices, [ap][(k1 k2)][(k1' k2')]; ap fastest in the loads
    for (int e = tid; e < APT * UL * UL; e += 256) {
        const int ap = e % APT, r = e / APT, ulp = r % UL, ul = r / UL;
        const int k1 = ul / K2, k2 = ul % K2, k1p = ulp / K2, k2p = ulp % K2;
        const int m2 = m20 + ap;
        Cm v = Cm(0);
        if (m2 < t.M2)
            v = (Cm)A[m1 * t.a_m1 + m2 * t.a_m2 + (long long)(k1 * K1 + k1p) * t.a_k1 + (long long)(k2 * K2 + k2p) * t.a_k2];
        Xs[(ap * UL + ul) * ULs + ulp] = v;
    }
    __syncthreads();
    const Cm* Tk = Ts;
    const Cm* Tb = Ts + (long long)d * UL * DRp;
    // Z_p[(k1 k2)][(n1' n2')] = sum_{(k1' k2')} X'[(k1 k2)][(k1' k2')] Tb_p[(k1' k2')][(n1' n2')]
    for (int w = tid; w < APT * d * UL; w += 256) {
        const int ul = w % UL, r = w / UL, ap = r % APT, p = r / APT;
        Cm acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = Cm(0);
        const Cm* xr = Xs + (ap * UL + ul) * ULs;
        const Cm* tb = Tb + (long long)p * UL * DRp;
        for (int k = 0; k < UL; ++k) {
            const Cm x = xr[k];
            const Cm* row = tb + k * DRp;
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4)
                if (4 * j4 < DR) {
                    Cm v[4];
                    lds4(row + 4 * j4, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[4 * j4 + q] = fma(x, v[q], acc[4 * j4 + q]);
                }
        }
        Cm* zr = Zs + (((long long)ap * d + p) * UL + ul) * DRp;
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4)
            if (4 * j4 < DRp) {
#pragma unroll
                for (int q = 0; q < 4; ++q) zr[4 * j4 + q] = acc[4 * j4 + q];
            }
    }
    __syncthreads();
    // Y[(n1 n1')][(n2 n2')] = sum_p sum_{(k1 k2)} Tk_p[(k1 k2)][(n1 n2)] Z_p[(k1 k2)][(n1' n2')],
    // staged as [ap][(n1 n1')][(n2 n2')] over the input matrices
    Cm* Os = Xs;
    for (int w = tid; w < APT * DR; w += 256) {
        const int dr = w % DR, ap = w / DR;
        Cm acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = Cm(0);
        for (int p = 0; p < d; ++p) {
            const Cm* tk = Tk + (long long)p * UL * DRp + dr;
            const Cm* zb = Zs + ((long long)ap * d + p) * UL * DRp;
            for (int k = 0; k < UL; ++k) {
                const Cm a = tk[k * DRp];
                const Cm* row = zb + k * DRp;
#pragma unroll
                for (int j4 = 0; j4 < 8; ++j4)
                    if (4 * j4 < DR) {
                        Cm v[4];
                        lds4(row + 4 * j4, v);
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[4 * j4 + q] = fma(a, v[q], acc[4 * j4 + q]);
                    }
            }
        }
        // the pad columns of Z are zero, so acc[j >= DR] is never stored
        const int n1 = dr / N2, n2 = dr % N2;
        Cm* orow = Os + (long long)ap * DR * DR;
        int n1p = 0, n2p = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < DR) {
                orow[(n1 * N1 + n1p) * (N2 * N2) + n2 * N2 + n2p] = acc[j];
                if (++n2p == N2) {
                    n2p = 0;
                    ++n1p;
                }
            }
    }
    __syncthreads();
    double* __restrict__ C = (double*)t.C;
    const int DR2 = DR * DR, N22 = N2 * N2;
    for (int e = tid; e < APT * DR2; e += 256) {
        const int ap = e / DR2, rem = e % DR2, i1 = rem / N22, i2 = rem % N22;
        const int m2 = m20 + ap;
        if (m2 >= t.M2) continue;
        const long long o = m1 * t.c_m1 + m2 * t.c_m2 + i1 * t.c_n1 + i2 * t.c_n2;
        const double r = (double)Os[e];
        C[o] = t.accumulate ? C[o] + r : r;
    }
}

size_t layer_smem_bytes(int d, int UL, int DR, bool f32) {
    const int apt = f32 ? LAYER_APT_F32 : LAYER_APT_F64;
    const long long DRp = layer_drp(DR), ULs = layer_uls(UL);
    const long long el = layer_round4(2LL * d * UL * DRp) +
                         layer_round4(std::max((long long)apt * UL * ULs, (long long)apt * DR * DR)) +
                         (long long)apt * d * UL * DRp;
    return (size_t)el * (f32 ? sizeof(float) : sizeof(double));
}

cudaError_t layer_prepare() {
    static std::mutex mu;
    std::lock_guard<std::mutex> guard(mu);
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_layer_pair<float, LAYER_APT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)LAYER_SMEM_MAX)))
        return e;
    if ((e = cudaFuncSetAttribute(k_layer_pair<double, LAYER_APT_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)LAYER_SMEM_MAX)))
        return e;
    done[dev] = true;
    return cudaSuccess;
}

cudaError_t launch_gcontract(const GTask* d_tasks, int ntasks, int max_tiles, bool cplx, cudaStream_t s, int mode,
                             long long smem_bytes) {
    if (ntasks <= 0) return cudaSuccess;
    dim3 grid(max_tiles, ntasks);
    const bool small = mode & 1;
    if (mode & GC_LAYER) {
        if (cplx || smem_bytes <= 0 || smem_bytes > (long long)LAYER_SMEM_MAX) return cudaErrorInvalidValue;
        if (mode & GC_F32)
            k_layer_pair<float, LAYER_APT_F32><<<grid, 256, (size_t)smem_bytes, s>>>(d_tasks);
        else
            k_layer_pair<double, LAYER_APT_F64><<<grid, 256, (size_t)smem_bytes, s>>>(d_tasks);
        return cudaGetLastError();
    }
    if (mode & GC_F32) {
        if (small) {
            if (cplx)
                k_gcontract_small<double2, float2><<<grid, 256, 0, s>>>(d_tasks);
            else
                k_gcontract_small<double, float><<<grid, 256, 0, s>>>(d_tasks);
        } else if (cplx) {
            k_gcontract<double2, float2><<<grid, 256, 0, s>>>(d_tasks);
        } else {
            // 128 x 64 tiles: at most as many as the 64 x 64 tiles max_tiles counts
            k_gcontract_f32w<<<grid, 256, 0, s>>>(d_tasks);
        }
        return cudaGetLastError();
    }
    if (small) {
        if (cplx)
            k_gcontract_small<double2><<<grid, 256, 0, s>>>(d_tasks);
        else
            k_gcontract_small<double><<<grid, 256, 0, s>>>(d_tasks);
    } else if (cplx) {
        k_gcontract<double2><<<grid, 256, 0, s>>>(d_tasks);
    } else {
        k_gcontract<double><<<grid, 256, 0, s>>>(d_tasks);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Householder QR / LQ
// Column j: alpha = x_j, x' = x_{j+1..m-1}, nrm = sqrt(|alpha|^2 + ||x'||^2),
// beta_j = -phase(alpha) nrm (no cancellation).  The reflector is kept in the scaled form
// H_j = I - tau_j v_j v_j^H with v_j = (x - beta_j e_j) / (alpha - beta_j), so v_j[j] = 1,
// |v_j[i]| <= 1 and tau_j = 1 + |alpha| / nrm in [1, 2]: nothing overflows however small the
// column is (the unscaled coefficient 1 / (nrm (nrm + |alpha|)) does once nrm is below
// ~1e-154, which happens to columns beyond the numerical rank).  ||x'|| is accumulated
// unscaled and recomputed relative to max |x'_i| when the sum is near underflow.  A column
// with x' = 0 gets H_j = I and beta_j = alpha.
// Q = H_0 ... H_{n-1} [I; 0]; finally column j is multiplied by phase(beta_j) so that
// R_jj = |beta_j| >= 0.  (k_qr_wy and k_qr_cluster below.)
constexpr int QR_MAXN = 512;
constexpr size_t QR_SMEM_LIMIT = 200 * 1024;
constexpr size_t QR32_SMEM_LIMIT = 100 * 1024;  // FP32 blocked QR: two CTAs per SM

// T of the compact-WY form of a panel (H_p0 ... H_p0+pw-1 = I - V T V^H, T upper triangular,
// T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] V[:, 0:j]^H v_j) from its reflectors in P:
// G = V^H V by the warps, then T column by column by thread 0.  The factorization and the Q
// phase both call it on the same reflectors, so both see the same T.
template <typename S, int NB, int NT>
__device__ __forceinline__ void panel_T(const S* P, int m, int p0, int pw, const typename ScalarTraits<S>::R* taus,
                                        S* G, S* Ts) {
    using R = typename ScalarTraits<S>::R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int pr = warp; pr < pw * pw; pr += NT / 32) {
        const int r = pr / pw, c = pr - r * pw;
        if (r >= c) continue;
        const S* vr = P + (size_t)r * m;
        const S* vc = P + (size_t)c * m;
        S d = zero<S>();
        for (int i = p0 + c + lane; i < m; i += 32) mac(d, conjv(vr[i]), vc[i]);  // v_c is zero above row p0+c
        d = warp_sum(d);
        if (lane == 0) G[r + c * NB] = d;
    }
    __syncthreads();
    if (tid == 0) {
        for (int c = 0; c < pw; ++c) {
            const R tc = taus[p0 + c];
            for (int r = 0; r < c; ++r) {
                S acc = zero<S>();
                for (int q = r; q < c; ++q) mac(acc, Ts[r + q * NB], G[q + c * NB]);
                Ts[r + c * NB] = scal(acc, -tc);
            }
            Ts[c + c * NB] = from_real<S>(tc);
            for (int r = c + 1; r < NB; ++r) Ts[r + c * NB] = zero<S>();
        }
        for (int c = pw; c < NB; ++c)
            for (int r = 0; r < NB; ++r) Ts[r + c * NB] = zero<S>();
    }
    __syncthreads();
}

// acc[r] += sum conj(P[r*m + i]) c[i] over the lane's rows i = p0 + lane + 32 j (V^H c for a
// panel of pw reflectors), the column read four rows at a time so that four loads are in
// flight (it lives in global memory); each acc[r] still adds its terms in row order.
template <typename S, int NB>
__device__ __forceinline__ void panel_dot(S (&acc)[NB], const S* c, const S* P, int m, int p0, int pw, int lane) {
    int i = p0 + lane;
    for (; i + 96 < m; i += 128) {
        const S x0 = c[i], x1 = c[i + 32], x2 = c[i + 64], x3 = c[i + 96];
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (r < pw) {
                const S* pr = P + (size_t)r * m + i;
                mac(acc[r], conjv(pr[0]), x0);
                mac(acc[r], conjv(pr[32]), x1);
                mac(acc[r], conjv(pr[64]), x2);
                mac(acc[r], conjv(pr[96]), x3);
            }
    }
    for (; i < m; i += 32) {
        const S x = c[i];
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (r < pw) mac(acc[r], conjv(P[(size_t)r * m + i]), x);
    }
}
// c[i] += sum_r P[r*m + i] w[r] over the lane's rows (c <- c + V w), four rows at a time; each
// element adds its terms in the order r = 0, 1, ...
template <typename S, int NB>
__device__ __forceinline__ void panel_update(S* c, const S* P, const S (&w)[NB], int m, int p0, int pw, int lane) {
    int i = p0 + lane;
    for (; i + 96 < m; i += 128) {
        S x[4] = {c[i], c[i + 32], c[i + 64], c[i + 96]};
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (r < pw) {
                const S* pr = P + (size_t)r * m + i;
#pragma unroll
                for (int q = 0; q < 4; ++q) mac(x[q], pr[32 * q], w[r]);
            }
#pragma unroll
        for (int q = 0; q < 4; ++q) c[i + 32 * q] = x[q];
    }
    for (; i < m; i += 32) {
        S x = c[i];
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (r < pw) mac(x, P[(size_t)r * m + i], w[r]);
        c[i] = x;
    }
}

// ---------------------------------------------------------------- blocked Householder QR
// For matrices too large for the cluster QR's shared memory (the (chi K) x chi site matrices
// at D=5, chi=96: 2400 x 96): one CTA per matrix, the matrix in the task's global workspace,
// taken in panels of NB columns (LAPACK's blocked Householder QR, in compact WY form):
//  * the panel (rows p0.., NB columns) is factored in shared memory with the reflectors
//    described above (scaled form v_j[j] = 1, tau_j in [1, 2]);
//  * its product H_p0 ... H_p0+nb-1 = I - V T V^H (T upper triangular, T_jj = tau_j,
//    T[0:j, j] = -tau_j T[0:j, 0:j] V[:, 0:j]^H v_j) is applied to every trailing column c as
//    c <- c - V (T^H (V^H c)), one column per warp in two passes with nb accumulators per
//    lane: each trailing column crosses the memory system three times per panel instead of
//    three times per column, and the FP64 units work on nb independent chains;
//  * Q = H_0 ... H_{n-1} [I; 0] is accumulated backwards, panel by panel, in place: the
//    panel's V is staged in shared memory, its columns of W are reset to e_k, and
//    c <- c - V (T (V^H c)) is applied to the columns k >= p0 (rows < p0 stay zero).
// Every reflector is the Householder reflector of its column (the one the unblocked order
// would form), so the result is the same Q up to rounding.  W occupies the first m*n scalars
// of the workspace; each panel's T is formed again in the Q phase rather than stored.
// S = float / float2 is the same algorithm in FP32 arithmetic, for the reduced-precision paths
// (tasks with in_float == 2, whose input is already an FP32 contraction result): on GB300 an
// FP32 instruction issues at 64 times the FP64 rate, and a single-CTA FP64 QR of a 2400 x 96
// site matrix is bound by exactly that rate.  Q is still written in FP64 (and the low-precision
// copy), and the loss is still summed in FP64.
template <typename S, int NB, int NT>
__global__ void __launch_bounds__(NT, NT == 512 ? 2 : 1) k_qr_wy(const QRTask* __restrict__ tasks) {
    using R = typename ScalarTraits<S>::R;
    using SW = typename ScalarTraits<S>::Wide;
    const QRTask& t = tasks[blockIdx.x];
    if (t.active && *t.active == 0) return;
    extern __shared__ __align__(16) unsigned char qr_smem[];
    S* P = (S*)qr_smem;  // panel, column c at P + c*m (absolute row index)
    __shared__ S betas[QR_MAXN];
    __shared__ R taus[QR_MAXN];
    __shared__ S Ts[NB * NB];  // T of the current panel, Ts[r + c*NB]
    __shared__ S G[NB * NB];   // V^H V of the panel
    __shared__ double redd[32];
    __shared__ R redr[32];
    const int m = t.m, n = t.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    S* W = (S*)t.work;
    double ss = 0.0;  // the loss -||in||^2, summed in FP64
    if constexpr (std::is_same<R, double>::value) {
        for (long long idx = tid; idx < (long long)m * n; idx += NT) {
            const int i = (int)(idx % m), j = (int)(idx / m);
            const long long src = (long long)i * t.in_rs + (long long)j * t.in_cs;
            S v = t.in_float ? from_float<S>(((const float*)t.in), src) : from_double<S>(t.in, src);
            if (t.conj_io) v = conjv(v);
            W[(size_t)j * m + i] = v;
            ss += abs2(v);
        }
    } else {
        // FP32 arithmetic: the matrix is scaled by 2^-e (exact), 2^(e-1) <= max |component| <
        // 2^e, so that no sum of squares overflows or underflows wholesale; Q does not change
        // and the loss is scaled back by 4^e.  Squares are summed in FP32 in runs of 16, the
        // runs in FP64.
        R amax = R(0);
        for (long long idx = tid; idx < (long long)m * n; idx += NT) {
            const int i = (int)(idx % m), j = (int)(idx / m);
            const long long src = (long long)i * t.in_rs + (long long)j * t.in_cs;
            S v = t.in_float ? from_float<S>(((const float*)t.in), src) : from_double<S>(t.in, src);
            if (t.conj_io) v = conjv(v);
            W[(size_t)j * m + i] = v;
            amax = max_r(amax, max_component(v));
        }
        amax = block_max(amax, redr);
        int e = 0;
        if (amax > R(0) && amax <= 3.4e38f) frexpf(amax, &e);
        const R sc = ldexpf(1.0f, -e);
        R part = R(0);
        int cnt = 0;
        for (long long idx = tid; idx < (long long)m * n; idx += NT) {
            const int i = (int)(idx % m), j = (int)(idx / m);
            const S v = scal(W[(size_t)j * m + i], sc);
            W[(size_t)j * m + i] = v;
            part += abs2(v);
            if (++cnt == 16) {
                ss += (double)part;
                part = R(0);
                cnt = 0;
            }
        }
        ss = ldexp(ss + (double)part, 2 * e);
    }
    ss = block_sum(ss, redd);
    if (tid == 0 && t.loss) *t.loss = -ss;
    __syncthreads();
    // ---- factorization
    for (int p0 = 0; p0 < n; p0 += NB) {
        const int pw = min(NB, n - p0), rows = m - p0;
        for (int idx = tid; idx < pw * rows; idx += NT) {
            const int c = idx / rows, i = p0 + (idx - c * rows);
            P[(size_t)c * m + i] = W[(size_t)(p0 + c) * m + i];
        }
        __syncthreads();
        for (int c = 0; c < pw; ++c) {
            const int j = p0 + c;
            S* col = P + (size_t)c * m;
            R xs2 = R(0);
            for (int i = j + 1 + tid; i < m; i += NT) xs2 += abs2(col[i]);
            xs2 = block_sum(xs2, redr);
            R xnorm = sqrt_r(xs2);
            if (xs2 < ScalarTraits<S>::tiny2()) {  // near underflow (uniform branch): rescale by max |x'_i|
                R amax = R(0);
                for (int i = j + 1 + tid; i < m; i += NT) amax = max_r(amax, absv(col[i]));
                amax = block_max(amax, redr);
                R t2 = R(0);
                if (amax > R(0))
                    for (int i = j + 1 + tid; i < m; i += NT) t2 += abs2(divr(col[i], amax));
                t2 = block_sum(t2, redr);
                xnorm = amax > R(0) ? amax * sqrt_r(t2) : R(0);
            }
            const S alpha = col[j];
            const R aa = absv(alpha);
            S beta = alpha;
            R tau = R(0);
            if (xnorm > R(0)) {
                const R nrm = hypot_r(aa, xnorm);
                const S ph = aa > R(0) ? divr(alpha, aa) : one<S>();
                beta = scal(ph, -nrm);
                tau = R(1) + aa / nrm;
                const R den = aa + nrm;  // |alpha - beta|
                const S cph = conjv(ph);
                if (den > ScalarTraits<S>::tiny_div()) {
                    const S sc = scal(cph, R(1) / den);
                    for (int i = j + 1 + tid; i < m; i += NT) col[i] = mul(col[i], sc);
                } else {
                    for (int i = j + 1 + tid; i < m; i += NT) col[i] = divr(mul(col[i], cph), den);
                }
            }
            __syncthreads();  // every thread has read alpha
            if (tid == 0) {
                betas[j] = beta;
                taus[j] = tau;
                col[j] = one<S>();  // v_j[j] = 1 (with tau = 0 the reflector is the identity)
            }
            for (int i = p0 + tid; i < j; i += NT) col[i] = zero<S>();  // V is zero above its diagonal
            __syncthreads();
            if (tau != R(0)) {  // H_j on the panel's later columns, one warp each
                for (int k = c + 1 + warp; k < pw; k += NT / 32) {
                    S* ck = P + (size_t)k * m;
                    S d0 = zero<S>(), d1 = zero<S>();
                    int i = j + lane;
                    for (; i + 32 < m; i += 64) {
                        mac(d0, conjv(col[i]), ck[i]);
                        mac(d1, conjv(col[i + 32]), ck[i + 32]);
                    }
                    if (i < m) mac(d0, conjv(col[i]), ck[i]);
                    const S f = scal(warp_sum(add(d0, d1)), -tau);
                    for (int r = j + lane; r < m; r += 32) mac(ck[r], col[r], f);
                }
            }
            __syncthreads();
        }
        // T of the panel (recomputed by the Q phase from the same reflectors)
        panel_T<S, NB, NT>(P, m, p0, pw, taus, G, Ts);
        // trailing columns: c <- c - V (T^H (V^H c)), one column per warp
        for (int k = p0 + pw + warp; k < n; k += NT / 32) {
            S* ck = W + (size_t)k * m;
            S acc[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) acc[r] = zero<S>();
            panel_dot<S, NB>(acc, ck, P, m, p0, pw, lane);
#pragma unroll
            for (int r = 0; r < NB; ++r) acc[r] = warp_sum(acc[r]);
            S wv[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                S a = zero<S>();
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q <= r) mac(a, conjv(Ts[q + r * NB]), acc[q]);  // (T^H w)_r
                wv[r] = scal(a, R(-1));
            }
            panel_update<S, NB>(ck, P, wv, m, p0, pw, lane);
        }
        // the panel's reflectors back to W (read again by the Q phase)
        for (int idx = tid; idx < pw * rows; idx += NT) {
            const int c = idx / rows, i = p0 + (idx - c * rows);
            W[(size_t)(p0 + c) * m + i] = P[(size_t)c * m + i];
        }
        __syncthreads();
    }
    // ---- Q, backwards over the panels, in place
    for (int p0 = ((n - 1) / NB) * NB; p0 >= 0; p0 -= NB) {
        const int pw = min(NB, n - p0), rows = m - p0;
        for (int idx = tid; idx < pw * rows; idx += NT) {
            const int c = idx / rows, i = p0 + (idx - c * rows);
            P[(size_t)c * m + i] = W[(size_t)(p0 + c) * m + i];
        }
        __syncthreads();
        panel_T<S, NB, NT>(P, m, p0, pw, taus, G, Ts);
        for (int idx = tid; idx < pw * m; idx += NT) {  // columns p0.. of the panel start as e_k
            const int c = idx / m, i = idx - c * m;
            W[(size_t)(p0 + c) * m + i] = i == p0 + c ? one<S>() : zero<S>();
        }
        __syncthreads();
        for (int k = p0 + warp; k < n; k += NT / 32) {
            S* ck = W + (size_t)k * m;
            S acc[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) acc[r] = zero<S>();
            panel_dot<S, NB>(acc, ck, P, m, p0, pw, lane);
#pragma unroll
            for (int r = 0; r < NB; ++r) acc[r] = warp_sum(acc[r]);
            S wv[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                S a = zero<S>();
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q >= r && q < pw) mac(a, Ts[r + q * NB], acc[q]);  // (T w)_r
                wv[r] = scal(a, R(-1));
            }
            panel_update<S, NB>(ck, P, wv, m, p0, pw, lane);
        }
        __syncthreads();
    }
    // ---- output: column k times phase(beta_k), so that R_kk = |beta_k| >= 0
    SW* out = (SW*)t.out;  // FP64 (complex-FP64) in every arithmetic
    for (long long idx = tid; idx < (long long)m * n; idx += NT) {
        const int i = (int)(idx % m), k = (int)(idx / m);
        const R bb = absv(betas[k]);
        const S ph = bb > R(0) ? divr(betas[k], bb) : one<S>();
        S vs = mul(W[(size_t)k * m + i], ph);
        if (t.conj_io) vs = conjv(vs);
        const SW v = widen(vs);
        out[(long long)i * t.out_rs + (long long)k * t.out_cs] = v;
        if (t.out2) {
            const int M2 = t.out2_M2 > 1 ? t.out2_M2 : 1, i1 = i / M2;
            store_split(t.out2, (long long)i1 * t.out2_rs + (long long)(i - i1 * M2) * t.out2_rs2 + (long long)k * t.out2_cs,
                        t.out2_kind, v, t.out2_x3, t.out2_kseg);
        }
    }
}

// Panel width of the blocked QR: the widest of 16, 8, 4, 2, 1 whose panel (nb x m scalars)
// fits QR_SMEM_LIMIT.
static int qr_wy_nb(int max_m, size_t ss) {
    int nb = 16;
    while (nb > 1 && (size_t)nb * max_m * ss > QR_SMEM_LIMIT) nb >>= 1;
    return nb;
}

// The QR with one task spread over a thread-block cluster of C CTAs (1 <= C <= 8), W and Q
// in shared memory.  On GB300 every warp-wide FP64 instruction occupies its SM sub-partition's
// FP64 unit for 64 cycles, however many lanes are active, and a square root or division is
// about ten such instructions.  So the cost of a Householder QR of these sizes is its count
// of FP64 instructions: along the per-column critical chain (the next column's update, its
// norm, the reflector's scalars) and per sub-partition for the bulk updates.  This form:
//  * column j belongs to CTA j % C, which keeps its columns of W in shared memory;
//  * in step j, warps 0-3 of the CTA owning column j+1 (one warp per sub-partition, rows
//    split between them) apply H_j to that column, form the reflector v_{j+1} from it and
//    publish it on a split cluster barrier; only then do that CTA's eight warps apply H_j
//    to its remaining columns, while every other CTA does so at once (each step begins
//    with a CTA barrier, so that no warp reads a column another is still updating);
//  * the reflector's square root and reciprocal are FP32 seeds refined by one third-order
//    step in FP64 (a handful of FP64 instructions instead of about thirty);
//  * the bulk updates take two columns per warp with one shared reduction tree;
//  * Q is formed column by column, Q e_k = H_0 H_1 ... H_k e_k, with the columns dealt to
//    the sub-partitions in snake order (balanced work) and no barrier, each v_j read from
//    its owner (distributed shared memory).
// The arithmetic on a column does not depend on which CTA or warp performs it, so the result
// is the same for every C.
// Shared memory per CTA: u (2 x m) | W (m x nl) | Q (m x nl) | tau (n) | all taus (n) |
// beta (n) | partial norm.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// named barrier 1: the four chain warps
__device__ __forceinline__ void chain_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 shfl_xor(double2 v, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
// Butterfly sum over the warp: every lane ends with the same total.
template <typename S>
__device__ __forceinline__ S warp_tree(S x) {
    for (int o = 16; o > 0; o >>= 1) x = add(x, shfl_xor(x, o));
    return x;
}
// Two sums in one tree: lanes < 16 end with the warp total of a, lanes >= 16 with that of b.
template <typename S>
__device__ __forceinline__ S pair_tree(S a, S b) {
    const bool lo = (threadIdx.x & 31) < 16;
    S x = add(lo ? a : b, shfl_xor(lo ? b : a, 16));
    for (int o = 8; o > 0; o >>= 1) x = add(x, shfl_xor(x, o));
    return x;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// x or -x by the sign bit (an integer operation, no FP64 instruction)
__device__ __forceinline__ double flip(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}
// alpha / |alpha| (1 for alpha = 0)
__device__ __forceinline__ double phase_of(double a, double aa) { return aa > 0.0 && a < 0.0 ? -1.0 : 1.0; }
__device__ __forceinline__ double2 phase_of(double2 a, double aa) { return aa > 0.0 ? divr(a, aa) : one<double2>(); }
__device__ __forceinline__ double apply_phase(double x, double ph) { return flip(x, ph < 0.0); }
__device__ __forceinline__ double2 apply_phase(double2 x, double2 ph) { return mul(x, ph); }

// 1/sqrt(s), s in [2^-100, 2^100]: the FP32 estimate y (relative error < 2^-21) refined by one
// step of Householder's third-order iteration for s^(-1/2), y (1 + e/2 + 3e^2/8) with
// e = 1 - s y^2 (remaining relative error ~ e^3, below FP64 rounding).
__device__ __forceinline__ double rsqrt_refined(double s) {
    const double y = (double)rsqrtf((float)s);
    const double e = fma(-(s * y), y, 1.0);
    return fma(y * fma(0.375, e, 0.5), e, y);
}
// 1/d, d in [2^-100, 2^100]: the FP32 reciprocal r refined by r (1 + e + e^2), e = 1 - d r
// (the third-order Newton-Raphson iteration for 1/d).
__device__ __forceinline__ double rcp_refined(double d) {
    const double r = (double)__frcp_rn((float)d);
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

__global__ void k_scalar_selftest(const double* __restrict__ x, long long n, double* rs, double* rc, double* rs_ref,
                                  double* rc_ref) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        rs[i] = rsqrt_refined(v);
        rc[i] = rcp_refined(v);
        rs_ref[i] = 1.0 / sqrt(v);
        rc_ref[i] = 1.0 / v;
    }
}
cudaError_t launch_scalar_selftest(const double* x, long long n, double* rsqrt_ours, double* rcp_ours,
                                   double* rsqrt_cuda, double* rcp_cuda, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long b = std::min<long long>((n + 255) / 256, 1024);
    k_scalar_selftest<<<(unsigned)b, 256, 0, s>>>(x, n, rsqrt_ours, rcp_ours, rsqrt_cuda, rcp_cuda);
    return cudaGetLastError();
}

// One warp: c <- c - tau v (v^H c) on rows >= j for c1 and, if c2 != nullptr, c2 (v may live
// in another CTA's shared memory).  A call is bound by the latency of its dependent FP64
// operations (each fed from shared memory), not by FP64 throughput, so a second column rides
// along almost for free: the two dot products share one reduction tree.  Each sums its rows
// in ascending order, so the result for a column does not depend on whether it is passed as
// c1 or c2.
template <typename S>
__device__ void warp_apply2(S* c1, S* c2, const S* v, double tau, int j, int m) {
    const int lane = threadIdx.x & 31;
    S a = zero<S>(), b = zero<S>();
    for (int i = j + lane; i < m; i += 32) {
        const S x = conjv(v[i]);
        mac(a, x, c1[i]);
        if (c2) mac(b, x, c2[i]);
    }
    const S f = scal(pair_tree(a, b), -tau);
    const S f1 = shfl_idx(f, 0), f2 = shfl_idx(f, 16);
    for (int i = j + lane; i < m; i += 32) {
        const S x = v[i];
        mac(c1[i], x, f1);
        if (c2) mac(c2[i], x, f2);
    }
    __syncwarp();
}

// Scratch of the chain warps (static shared memory).
template <typename S>
struct ChainScratch {
    S dot[4];
    double nrm[4];
    double amax[4];
    S alpha;
};

// Warps 0-3 of the CTA owning column nxt: if tau != 0, apply H_j (v_j in ub) to column c on
// rows >= j; then turn c into the scaled reflector v_nxt in place (v_nxt[nxt] = 1; see above
// for the scaled form) and record tau_nxt, beta_nxt.  Warp w takes the rows
// base + 32 (4 t + w) + lane, base = j (nxt when there is no H_j).
template <typename S>
__device__ void chain_reflector(S* c, const S* ub, double tau, int j, int nxt, int m, ChainScratch<S>& cs,
                                double* taus, S* betas) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = tau != 0.0 ? j : nxt;
    double p = 0.0;
    if (tau != 0.0) {
        S a = zero<S>();
        for (int i = base + 32 * w + lane; i < m; i += 128) mac(a, conjv(ub[i]), c[i]);
        a = warp_tree(a);
        if (lane == 0) cs.dot[w] = a;
        chain_sync();
        const S f = scal(add(add(cs.dot[0], cs.dot[1]), add(cs.dot[2], cs.dot[3])), -tau);
        for (int i = base + 32 * w + lane; i < m; i += 128) {
            S x = c[i];
            mac(x, ub[i], f);
            c[i] = x;
            if (i > nxt) p += abs2(x);
        }
    } else {
        for (int i = base + 32 * w + lane; i < m; i += 128)
            if (i > nxt) p += abs2(c[i]);
    }
    if (w == 0 && lane == nxt - base) cs.alpha = c[nxt];  // row nxt lies in warp 0's first block
    p = warp_tree(p);
    if (lane == 0) cs.nrm[w] = p;
    chain_sync();
    const double xs2 = (cs.nrm[0] + cs.nrm[1]) + (cs.nrm[2] + cs.nrm[3]);
    const S alpha = cs.alpha;
    const double aa = absv(alpha);
    double nrm = 0.0, tau_n = 0.0, rd = 0.0;
    bool any = true;
    if (xs2 < 1e-280) {  // near underflow (uniform branch): rescale by max |x'_i|
        double am = 0.0;
        for (int i = base + 32 * w + lane; i < m; i += 128)
            if (i > nxt) am = fmax(am, absv(c[i]));
        am = warp_max(am);
        if (lane == 0) cs.amax[w] = am;
        chain_sync();
        am = fmax(fmax(cs.amax[0], cs.amax[1]), fmax(cs.amax[2], cs.amax[3]));
        double t2 = 0.0;
        if (am > 0.0)
            for (int i = base + 32 * w + lane; i < m; i += 128)
                if (i > nxt) t2 += abs2(divr(c[i], am));
        t2 = warp_tree(t2);
        chain_sync();  // every warp has read cs.nrm and cs.amax
        if (lane == 0) cs.nrm[w] = t2;
        chain_sync();
        t2 = (cs.nrm[0] + cs.nrm[1]) + (cs.nrm[2] + cs.nrm[3]);
        any = am > 0.0;
        if (any) {
            nrm = hypot(aa, am * sqrt(t2));
            tau_n = 1.0 + aa / nrm;
            rd = 1.0 / (aa + nrm);
        }
    } else {
        const double s = fma(aa, aa, xs2);
        if (s >= 0x1p-100 && s <= 0x1p100) {
            const double y = rsqrt_refined(s);
            nrm = s * y;
            tau_n = fma(aa, y, 1.0);
            rd = rcp_refined(aa + nrm);
        } else {
            nrm = (aa < 1e150 && xs2 < 1e300) ? sqrt(s) : hypot(aa, sqrt(xs2));
            tau_n = 1.0 + aa / nrm;
            rd = 1.0 / (aa + nrm);
        }
    }
    S beta = alpha;
    if (any) {
        const S ph = phase_of(alpha, aa);
        beta = apply_phase(from_real<S>(flip(nrm, true)), ph);  // -phase(alpha) nrm
        const S sc = apply_phase(from_real<S>(rd), conjv(ph));
        for (int i = base + 32 * w + lane; i < m; i += 128)
            if (i > nxt) c[i] = mul(c[i], sc);
        if (w == 0 && lane == nxt - base) c[nxt] = one<S>();
    }
    if (w == 0 && lane == 0) {
        taus[nxt] = any ? tau_n : 0.0;
        betas[nxt] = beta;
    }
    __syncwarp();
}

template <typename S>
__global__ void __launch_bounds__(256) k_qr_cluster(const QRTask* __restrict__ tasks, int C) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const QRTask& t = tasks[blockIdx.x / C];
    if (t.active && *t.active == 0) return;  // uniform over the cluster
    const int m = t.m, n = t.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nl = (n - rank + C - 1) / C;   // local columns j = rank + lc * C
    const int nlmax = (n + C - 1) / C;       // same layout in every CTA of the cluster
    extern __shared__ __align__(16) unsigned char qr_smem[];
    S* u = (S*)qr_smem;  // two staging buffers of m entries
    S* W = u + 2 * m;
    S* Q = W + (size_t)m * nlmax;
    double* taus = (double*)(Q + (size_t)m * nlmax);
    double* tall = taus + QR_MAXN;
    S* betas = (S*)(tall + QR_MAXN);
    __shared__ S phs[QR_MAXN];
    __shared__ ChainScratch<S> cs;
    const S* in = (const S*)t.in;
    {
        // eight loads per thread in flight at a time (each is a round trip to L2)
        constexpr int LB = 8;
        const int total = m * nl;
        for (int base = 0; base < total; base += 256 * LB) {
            S v[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const int idx = base + q * 256 + tid;
                if (idx < total) {
                    const int lc = idx / m, i = idx - lc * m, j = rank + lc * C;
                    const long long src = (long long)i * t.in_rs + (long long)j * t.in_cs;
                    v[q] = t.in_float ? from_float<S>(((const float*)t.in), src) : in[src];
                }
            }
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const int idx = base + q * 256 + tid;
                if (idx < total) W[idx] = t.conj_io ? conjv(v[q]) : v[q];
            }
        }
    }
    if (t.loss) {  // uniform: squared column norms, for the loss -||A||^2 of the fit (App. A)
        __syncthreads();
        for (int lc = warp; lc < nl; lc += 8) {
            double p = 0.0;
            for (int i = lane; i < m; i += 32) p += abs2(W[(size_t)lc * m + i]);
            p = warp_tree(p);
            if (lane == 0) tall[lc] = p;  // tall is free until the R phase ends
        }
    }
    cluster.sync();  // W loaded everywhere; column norms published
    if (rank == 0 && warp == 0 && t.loss) {
        // summed over columns in a fixed order (lane j takes columns j, j + 32, ...), so that
        // the loss does not depend on how the columns are spread over the cluster
        double p = 0.0;
        for (int j = lane; j < n; j += 32) p += *cluster.map_shared_rank(tall + j / C, j % C);
        p = warp_tree(p);
        if (lane == 0) *t.loss = -p;
    }  // tall is rewritten only after the R phase, when every CTA is past this read
    // ---- R: phase p of the split cluster barrier publishes v_p and tau_p
    if (n > 0) {
        if (rank == 0 && warp < 4) chain_reflector(W, u, 0.0, 0, 0, m, cs, taus, betas);
        cluster_arrive();
    }
    for (int j = 0; j < n; ++j) {
        const int owner = j % C, nxt = j + 1;
        cluster_wait();  // v_j and tau_j are published
        const double tau = owner == rank ? taus[j] : *cluster.map_shared_rank(taus + j, owner);
        S* ub = u + (size_t)(j & 1) * m;
        const S* vj = W + (size_t)(j / C) * m;
        if (owner != rank) vj = cluster.map_shared_rank(vj, owner);
        const bool own_next = nxt < n && rank == nxt % C;
        // copied whatever tau is (unused when tau = 0), so that this read of the owner's shared
        // memory overlaps the read of tau instead of waiting for it
        for (int i = j + tid; i < m; i += 256) ub[i] = vj[i];
        __syncthreads();  // u holds v_j; every warp has finished step j-1
        if (own_next) {
            // the chain first; the bulk update of this CTA waits for it
            if (warp < 4) chain_reflector(W + (size_t)(nxt / C) * m, ub, tau, j, nxt, m, cs, taus, betas);
            __syncthreads();
        }
        if (nxt < n) cluster_arrive();
        if (tau != 0.0) {
            // local columns k > j, without column j+1 on its owner: eight warps, two columns each
            const int lk0 = (nxt - rank + C - 1) / C + (own_next ? 1 : 0);
            for (int t0 = warp; lk0 + t0 < nl; t0 += 16) {
                const int l1 = lk0 + t0, l2 = l1 + 8;
                warp_apply2(W + (size_t)l1 * m, l2 < nl ? W + (size_t)l2 * m : (S*)nullptr, ub, tau, j, m);
            }
        }
    }
    cluster.sync();  // every reflector is final
    for (int jj = tid; jj < n; jj += 256) tall[jj] = jj % C == rank ? taus[jj] : *cluster.map_shared_rank(taus + jj, jj % C);
    for (int lc = tid; lc < nl; lc += 256) {  // phase(beta_k) of the local columns, so that R_kk >= 0
        const S b = betas[rank + lc * C];
        phs[lc] = phase_of(b, absv(b));
    }
    __syncthreads();
    // ---- Q: local columns in descending k; the eight longest get a warp each (warp t), the
    // next eight are dealt back from warp 7 to warp 0, and so on; each warp takes its
    // columns two at a time (a short column rides along with a long one)
    {
        int pend = -1;
        for (int q = 0; q <= nl; ++q) {
            int lc = -1;
            if (q < nl) {
                const int b = q >> 3, p = q & 7;
                if (((b & 1) ? 7 - p : p) != warp) continue;
                lc = nl - 1 - q;
                if (pend < 0) {
                    pend = lc;
                    continue;
                }
            }
            if (pend < 0) break;
            const int k1 = rank + pend * C, k2 = lc >= 0 ? rank + lc * C : -1;  // k1 > k2
            S* y1 = Q + (size_t)pend * m;
            S* y2 = lc >= 0 ? Q + (size_t)lc * m : nullptr;
            for (int i = lane; i < m; i += 32) {
                y1[i] = i == k1 ? one<S>() : zero<S>();
                if (y2) y2[i] = i == k2 ? one<S>() : zero<S>();
            }
            __syncwarp();
            for (int jj = k1; jj >= 0; --jj) {  // H_jj leaves e_k unchanged for jj > k
                const double tj = tall[jj];
                if (tj == 0.0) continue;
                const S* v = W + (size_t)(jj / C) * m;
                if (jj % C != rank) v = cluster.map_shared_rank(v, jj % C);
                warp_apply2(y1, jj <= k2 ? y2 : (S*)nullptr, v, tj, jj, m);
            }
            pend = -1;
        }
    }
    __syncthreads();
    S* out = (S*)t.out;
    for (int idx = tid; idx < m * nl; idx += 256) {
        const int lc = idx / m, i = idx - lc * m, k = rank + lc * C;
        S v = apply_phase(Q[idx], phs[lc]);
        if (t.conj_io) v = conjv(v);
        out[(long long)i * t.out_rs + (long long)k * t.out_cs] = v;
        if (t.out2) {
            const int M2 = t.out2_M2 > 1 ? t.out2_M2 : 1, i1 = i / M2;
            store_split(t.out2, (long long)i1 * t.out2_rs + (long long)(i - i1 * M2) * t.out2_rs2 + (long long)k * t.out2_cs,
                        t.out2_kind, v, t.out2_x3, t.out2_kseg);
        }
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

constexpr size_t QR_CLUSTER_SMEM = QR_SMEM_LIMIT + QR_MAXN * (16 + 16) + 16;

static int sm_count() {
    static std::atomic<int> cached{0};  // read by the server's worker and read-out threads
    int n = cached.load(std::memory_order_relaxed);
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cached.store(n, std::memory_order_relaxed);
    }
    return n;
}

static size_t qr_cluster_smem(int max_m, long long max_mn, int C, size_t ss) {
    // m * ceil(n / C) <= m * n / C + m
    const size_t cols = (size_t)(max_mn / C) + (size_t)max_m;
    return (2 * (size_t)max_m + 2 * cols) * ss + QR_MAXN * (16 + ss) + 16;
}

cudaError_t qr_prepare(int max_m, bool cplx) {
    static std::mutex mu;  // the request server reads out on a second thread
    std::lock_guard<std::mutex> guard(mu);
    // A kernel attribute applies to the current device only, so the state is kept per device.
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (qr_wy_nb(max_m, cplx ? sizeof(double2) : sizeof(double)) * (size_t)max_m * (cplx ? 16 : 8) > QR_SMEM_LIMIT)
        return cudaErrorInvalidValue;  // not even one column of this height fits shared memory
    if (done[dev][cplx ? 1 : 0]) return cudaSuccess;
    const int lim = (int)QR_SMEM_LIMIT;
    cudaError_t e;
    // the FP32-arithmetic blocked QR (reduced-precision paths): 512 threads, two CTAs per SM
    const int lim32 = (int)QR32_SMEM_LIMIT;
    if (cplx) {
        if ((e = cudaFuncSetAttribute(k_qr_wy<float2, 1, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<float2, 2, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<float2, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<float2, 8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
    } else {
        if ((e = cudaFuncSetAttribute(k_qr_wy<float, 1, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<float, 2, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<float, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<float, 8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim32))) return e;
    }
    if (cplx) {
        if ((e = cudaFuncSetAttribute(k_qr_cluster<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)QR_CLUSTER_SMEM)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double2, 1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double2, 2, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double2, 4, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double2, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double2, 16, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    } else {
        if ((e = cudaFuncSetAttribute(k_qr_cluster<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)QR_CLUSTER_SMEM)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double, 1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double, 2, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double, 4, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_qr_wy<double, 16, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    }
    done[dev][cplx ? 1 : 0] = true;
    return cudaSuccess;
}

bool qr_cluster_fits(int max_m, long long max_mn, bool cplx, int C) {
    return C >= 1 && C <= 8 && qr_cluster_smem(max_m, max_mn, C, cplx ? sizeof(double2) : sizeof(double)) <= QR_CLUSTER_SMEM;
}

cudaError_t launch_qr(const QRTask* d_tasks, int ntasks, int max_m, long long max_mn, bool cplx, cudaStream_t s,
                      int cluster) {
    if (ntasks <= 0) return cudaSuccess;
    if (cluster & QR_F32) {
        // FP32 arithmetic: the blocked QR, one CTA of 512 threads per task, whatever the size,
        // panels of up to 8 columns so that two CTAs share an SM (the one-CTA QR is bound by
        // latency, not by a unit's throughput)
        const size_t fsz = cplx ? sizeof(float2) : sizeof(float);
        int nb = 8;
        while (nb > 1 && (size_t)nb * max_m * fsz > QR32_SMEM_LIMIT) nb >>= 1;
        const size_t sm = (size_t)nb * max_m * fsz;
        if (sm > QR32_SMEM_LIMIT) return cudaErrorInvalidValue;
#define WY_CASE(NB_)                                                               \
        if (nb == NB_) {                                                           \
            if (cplx) k_qr_wy<float2, NB_, 512><<<ntasks, 512, sm, s>>>(d_tasks);  \
            else k_qr_wy<float, NB_, 512><<<ntasks, 512, sm, s>>>(d_tasks);        \
            return cudaGetLastError();                                             \
        }
        WY_CASE(8) WY_CASE(4) WY_CASE(2) WY_CASE(1)
#undef WY_CASE
        return cudaErrorInvalidValue;
    }
    cluster &= 0xFF;
    // Spread each task over C CTAs so that the launch covers the SMs (with at least two
    // columns per CTA), and over more CTAs if its matrix does not fit one CTA's shared memory.
    // cluster > 0 asks for that C (the autotuner's choice; the result is the same for every C).
    const size_t ssz = cplx ? sizeof(double2) : sizeof(double);
    const int n_est = (int)std::max<long long>(1, max_mn / std::max(1, max_m));
    int C = std::min(8, std::max(1, sm_count() / ntasks));
    C = std::max(1, std::min(C, n_est / 2));
    if (cluster > 0) C = std::min(8, cluster);
    while (C < 8 && qr_cluster_smem(max_m, max_mn, C, ssz) > QR_CLUSTER_SMEM) ++C;
    if (qr_cluster_smem(max_m, max_mn, C, ssz) <= QR_CLUSTER_SMEM) {
        const size_t sm = qr_cluster_smem(max_m, max_mn, C, ssz);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C * ntasks);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cplx ? cudaLaunchKernelEx(&cfg, k_qr_cluster<double2>, d_tasks, C)
                    : cudaLaunchKernelEx(&cfg, k_qr_cluster<double>, d_tasks, C);
    }
    // too large for the shared memory of a cluster: one CTA per task, the blocked QR with the
    // matrix in the task's global workspace and a panel of nb columns in shared memory
    const int nb = qr_wy_nb(max_m, ssz);
    const size_t sm = (size_t)nb * max_m * ssz;
    if (sm > QR_SMEM_LIMIT) return cudaErrorInvalidValue;
#define WY_CASE(NB_)                                                               \
    if (nb == NB_) {                                                               \
        if (cplx) k_qr_wy<double2, NB_, 256><<<ntasks, 256, sm, s>>>(d_tasks);          \
        else k_qr_wy<double, NB_, 256><<<ntasks, 256, sm, s>>>(d_tasks);                \
        return cudaGetLastError();                                                 \
    }
    WY_CASE(16) WY_CASE(8) WY_CASE(4) WY_CASE(2) WY_CASE(1)
#undef WY_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- random fill
__global__ void k_rand(const RandTask* __restrict__ tasks, unsigned long long seed, const int* sweep_ctr, int cplx) {
    const RandTask& t = tasks[blockIdx.y];
    const uint64_t stream = t.stream | (sweep_ctr ? ((uint64_t)(*sweep_ctr) << 36) : 0ull);
    const uint64_t key = rng_key(seed, stream);
    const long long cnt = cplx ? 2 * t.n : t.n;
    double* p = (double*)t.ptr;
    if (t.active && blockIdx.x == 0 && threadIdx.x == 0) *t.active = 1;
    if (t.warm && t.warm_ctr && *t.warm_ctr > 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
        p[i] = u_pm1(key, (uint64_t)i);
}
cudaError_t launch_rand(const RandTask* d_tasks, int ntasks, unsigned long long seed, const int* sweep_ctr,
                        bool cplx, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    k_rand<<<dim3(8, ntasks), 256, 0, s>>>(d_tasks, seed, sweep_ctr, cplx ? 1 : 0);
    return cudaGetLastError();
}

__global__ void k_set_int(int* p, int n, int v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}
cudaError_t launch_set_int(int* p, int n, int v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_set_int<<<(n + 255) / 256, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}
__global__ void k_add_int(int* p, int v) { *p += v; }
cudaError_t launch_add_int(int* p, int v, cudaStream_t s) {
    k_add_int<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fit stop rule (App. A)
// One CTA: every fit of the group tests std/|mean| of its sweep's losses; the loop
// continues while any fit is still active and fewer than loop->max sweeps have run.
__global__ void __launch_bounds__(256) k_check(const CheckTask* __restrict__ tasks, int ntasks, double tol, LoopDesc* loop) {
    int any = 0;
    for (int i = threadIdx.x; i < ntasks; i += blockDim.x) {
        const CheckTask& t = tasks[i];
        if (*t.active == 0) continue;
        *t.counter += 1;
        double mean = 0.0;
        for (int k = 0; k < t.count; ++k) mean += t.losses[k];
        mean /= t.count;
        double var = 0.0;
        for (int k = 0; k < t.count; ++k) {
            const double dv = t.losses[k] - mean;
            var += dv * dv;
        }
        const double sd = sqrt(var / t.count);
        if (mean != 0.0 && sd / fabs(mean) < tol) *t.active = 0;
        else any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0 && loop) {
        const int it = ++loop->iter;
        loop->total += 1;
        const unsigned int more = (any && it < loop->max) ? 1u : 0u;
        if (loop->use_handle) cudaGraphSetConditional((cudaGraphConditionalHandle)loop->handle, more);
    }
}
cudaError_t launch_check(const CheckTask* d_tasks, int ntasks, double tol, LoopDesc* loop, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    k_check<<<1, 256, 0, s>>>(d_tasks, ntasks, tol, loop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- scale to unit norm
template <typename S>
__global__ void __launch_bounds__(256) k_scale(const ScaleTask* __restrict__ tasks, int* status) {
    const ScaleTask& t = tasks[blockIdx.x];
    __shared__ double red[32];
    S* p = (S*)t.ptr;
    double ss = 0.0;
    for (long long i = threadIdx.x; i < t.n; i += 256) ss += abs2(p[i]);
    ss = block_sum(ss, red);
    if (!(ss > 0.0) || !isfinite(ss)) {
        if (threadIdx.x == 0) atomicExch(status, 1);
        return;
    }
    const double inv = 1.0 / sqrt(ss);
    for (long long i = threadIdx.x; i < t.n; i += 256) p[i] = scal(p[i], inv);
}
cudaError_t launch_scale(const ScaleTask* d_tasks, int ntasks, bool cplx, int* status, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    if (cplx)
        k_scale<double2><<<ntasks, 256, 0, s>>>(d_tasks, status);
    else
        k_scale<double><<<ntasks, 256, 0, s>>>(d_tasks, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- message assembly
template <typename S>
__global__ void __launch_bounds__(256) k_assemble(const AssembleTask* __restrict__ tasks) {
    const AssembleTask& t = tasks[blockIdx.x];
    const S c = mul(*(const S*)t.corner0, *(const S*)t.corner1);
    for (int s = 0; s < t.nsites; ++s) {
        const S* src = (const S*)t.src[s];
        S* dst = (S*)t.dst[s];
        for (long long i = threadIdx.x; i < t.size[s]; i += 256) dst[i] = (s == 0) ? mul(src[i], c) : src[i];
    }
}
cudaError_t launch_assemble(const AssembleTask* d_tasks, int ntasks, bool cplx, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    if (cplx)
        k_assemble<double2><<<ntasks, 256, 0, s>>>(d_tasks);
    else
        k_assemble<double><<<ntasks, 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- normalisation + residual term
// tau = <I|m>: per site the matrix sum_k m[a][k*D+k][b], chained left to right (on a
// single-layer network <1|m>: the sum over every k).
constexpr int NORM_MAXB = 1024;
template <typename S>
__global__ void __launch_bounds__(256) k_normalise(const NormTask* __restrict__ tasks) {
    const NormTask& t = tasks[blockIdx.x];
    __shared__ S v[NORM_MAXB], w[NORM_MAXB];
    if (threadIdx.x == 0) v[0] = one<S>();
    __syncthreads();
    int na = 1;
    for (int s = 0; s < t.nsites; ++s) {
        const S* m = (const S*)t.sites[s];
        const int A = t.a[s], K = t.k[s], B = t.b[s];
        for (int b = threadIdx.x; b < B; b += 256) {
            S acc = zero<S>();
            for (int a = 0; a < na; ++a) {
                if (t.ones)
                    for (int k = 0; k < K; ++k) mac(acc, v[a], m[((long long)a * K + k) * B + b]);
                else
                    for (int k = 0; k < t.D; ++k) mac(acc, v[a], m[((long long)a * K + (k * t.D + k)) * B + b]);
            }
            w[b] = acc;
        }
        __syncthreads();
        for (int b = threadIdx.x; b < B; b += 256) v[b] = w[b];
        na = B;
        (void)A;
        __syncthreads();
    }
    const S tau = v[0];
    const double mmr = *(const double*)t.mm;  // real part of <m|m>
    const S mo = *(const S*)t.mo;
    const double nrm = sqrt(fmax(mmr, 0.0));
    if (!(nrm > 0.0) || !isfinite(nrm)) {
        if (threadIdx.x == 0) {
            atomicExch(t.status, 1);
            *t.resid = 0.0;
        }
        return;
    }
    const double at = absv(tau);
    const S ph = at > 1e-14 * nrm ? scal(conjv(tau), 1.0 / at) : one<S>();
    const S sc = scal(ph, 1.0 / nrm);
    S* p = (S*)t.site0;
    for (long long i = threadIdx.x; i < t.size0; i += 256) p[i] = mul(p[i], sc);
    if (threadIdx.x == 0) {
        // <s m | m_old> = conj(s) <m|m_old>
        const S ov = mul(conjv(sc), mo);
        double re;
        if constexpr (sizeof(S) == sizeof(double)) re = *(const double*)&ov;
        else re = ((const double*)&ov)[0];
        *t.resid = 2.0 - 2.0 * re;
    }
}
cudaError_t launch_normalise(const NormTask* d_tasks, int ntasks, bool cplx, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    if (cplx)
        k_normalise<double2><<<ntasks, 256, 0, s>>>(d_tasks);
    else
        k_normalise<double><<<ntasks, 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

__global__ void k_mean(const double* in, int n, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += in[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = n > 0 ? s / n : 0.0;
}
cudaError_t launch_mean(const double* in, int n, double* out, cudaStream_t s) {
    k_mean<<<1, 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- double layer (Fig. 1(a,b))
template <typename S>
__global__ void k_double_layer(const DLTask* __restrict__ tasks) {
    const DLTask& t = tasks[blockIdx.y];
    const int Ku = t.Du * t.Du, Kl = t.Dl * t.Dl, Kd = t.Dd * t.Dd, Kr = t.Dr * t.Dr;
    const long long total = (long long)Ku * Kl * Kd * Kr;
    const long long vol = (long long)t.Du * t.Dl * t.Dd * t.Dr;
    const S* T = (const S*)t.T;
    const S* O = (const S*)t.O;
    S* E = (S*)t.E;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int ir = (int)(r % Kr); r /= Kr;
        const int id = (int)(r % Kd); r /= Kd;
        const int il = (int)(r % Kl); r /= Kl;
        const int iu = (int)r;
        const int u = iu / t.Du, u2 = iu % t.Du, l = il / t.Dl, l2 = il % t.Dl;
        const int dd = id / t.Dd, d2 = id % t.Dd, rr = ir / t.Dr, r2 = ir % t.Dr;
        const long long ket = (((long long)u * t.Dl + l) * t.Dd + dd) * t.Dr + rr;
        const long long bra = (((long long)u2 * t.Dl + l2) * t.Dd + d2) * t.Dr + r2;
        S acc = zero<S>();
        for (int pp = 0; pp < t.d; ++pp) {
            // (O T)[p'] = sum_p O[p'][p] T[p]
            S ot = zero<S>();
            if (O) {
                for (int p = 0; p < t.d; ++p) mac(ot, O[pp * t.d + p], T[p * vol + ket]);
            } else {
                ot = T[pp * vol + ket];
            }
            mac(acc, ot, conjv(T[pp * vol + bra]));
        }
        E[e] = acc;
    }
}
cudaError_t launch_double_layer(const DLTask* d_tasks, int ntasks, long long max_out, bool cplx, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    long long bx = (max_out + 255) / 256;
    if (bx > 4096) bx = 4096;
    dim3 grid((unsigned)bx, ntasks);
    if (cplx)
        k_double_layer<double2><<<grid, 256, 0, s>>>(d_tasks);
    else
        k_double_layer<double><<<grid, 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

// Double layer in the Hermitian basis: T and O complex (O Hermitian or NULL), E real.
// Each merged leg index k = a*D + b is the V coordinate of the pair (a, b):
// a == b -> v_(a,a); a < b -> (v_(a,b) + v_(b,a)) / sqrt 2; a > b -> (v_(b,a) - v_(a,b)) / (i sqrt 2),
// on the up and left legs; the down and right legs take conj(V) (the a > b coordinate
// changes sign).  Every bond joins a down (right) leg to an up (left) leg, and
// V^T conj(V) = I, so contractions over bonds are unchanged (V^T V alone would swap ket
// and bra).  E'[ku][kl][kd][kr] = Re sum over the (<= 2 per leg) pairs of the product of the
// leg coefficients times E^O at those pairs; the imaginary part vanishes for Hermitian O.
struct HbLeg {
    int ket[2], bra[2];
    double2 c[2];
    int n;
};
__device__ __forceinline__ HbLeg hb_leg(int k, int D, bool conj_basis) {
    HbLeg h;
    const int a = k / D, b = k % D;
    const double s = 0.70710678118654752440;
    if (a == b) {
        h.n = 1;
        h.ket[0] = a; h.bra[0] = a; h.c[0] = make_double2(1.0, 0.0);
    } else if (a < b) {
        h.n = 2;
        h.ket[0] = a; h.bra[0] = b; h.c[0] = make_double2(s, 0.0);
        h.ket[1] = b; h.bra[1] = a; h.c[1] = make_double2(s, 0.0);
    } else {
        h.n = 2;  // V: 1/(i sqrt 2) = -i/sqrt 2 on v_(b,a), +i/sqrt 2 on v_(a,b); conj(V): opposite
        const double sg = conj_basis ? -1.0 : 1.0;
        h.ket[0] = b; h.bra[0] = a; h.c[0] = make_double2(0.0, -s * sg);
        h.ket[1] = a; h.bra[1] = b; h.c[1] = make_double2(0.0, s * sg);
    }
    return h;
}
__global__ void k_double_layer_hb(const DLTask* __restrict__ tasks) {
    const DLTask& t = tasks[blockIdx.y];
    const int Ku = t.Du * t.Du, Kl = t.Dl * t.Dl, Kd = t.Dd * t.Dd, Kr = t.Dr * t.Dr;
    const long long total = (long long)Ku * Kl * Kd * Kr;
    const long long vol = (long long)t.Du * t.Dl * t.Dd * t.Dr;
    const double2* T = (const double2*)t.T;
    const double2* O = (const double2*)t.O;
    double* E = (double*)t.E;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int ir = (int)(r % Kr); r /= Kr;
        const int id = (int)(r % Kd); r /= Kd;
        const int il = (int)(r % Kl); r /= Kl;
        const int iu = (int)r;
        const HbLeg hu = hb_leg(iu, t.Du, false), hl = hb_leg(il, t.Dl, false);
        const HbLeg hd = hb_leg(id, t.Dd, true), hr = hb_leg(ir, t.Dr, true);
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < hu.n; ++a)
            for (int b = 0; b < hl.n; ++b)
                for (int c = 0; c < hd.n; ++c)
                    for (int f = 0; f < hr.n; ++f) {
                        const long long ket = (((long long)hu.ket[a] * t.Dl + hl.ket[b]) * t.Dd + hd.ket[c]) * t.Dr + hr.ket[f];
                        const long long bra = (((long long)hu.bra[a] * t.Dl + hl.bra[b]) * t.Dd + hd.bra[c]) * t.Dr + hr.bra[f];
                        double2 v = make_double2(0.0, 0.0);
                        for (int pp = 0; pp < t.d; ++pp) {
                            double2 ot = make_double2(0.0, 0.0);
                            if (O) {
                                for (int p = 0; p < t.d; ++p) mac(ot, O[pp * t.d + p], T[p * vol + ket]);
                            } else {
                                ot = T[pp * vol + ket];
                            }
                            mac(v, ot, conjv(T[pp * vol + bra]));
                        }
                        const double2 cf = mul(mul(hu.c[a], hl.c[b]), mul(hd.c[c], hr.c[f]));
                        mac(acc, cf, v);
                    }
        E[e] = acc.x;
    }
}
cudaError_t launch_double_layer_hb(const DLTask* d_tasks, int ntasks, long long max_out, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    long long bx = (max_out + 255) / 256;
    if (bx > 4096) bx = 4096;
    dim3 grid((unsigned)bx, ntasks);
    k_double_layer_hb<<<grid, 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- initial messages
// One thread per message (a handful of sites of at most 256 entries each).
__device__ double init_entry(const MsgInitTask& t, uint64_t key, int k) {
    const int D = t.D;
    if (t.single) return t.mode == 0 ? 1.0 : (u_pm1(key, (uint64_t)k) + 1.0) * 0.5;
    const int a = k / D, b = k - a * D;
    if (t.mode == 0) return a == b ? 1.0 : 0.0;
    // site = G G^T with G[i][j] = sqrt(-2 log(1 - u1)) cos(2 pi u2), u1, u2 uniform in [0, 1)
    auto g = [&](int i, int j) {
        const uint64_t jj = (uint64_t)(i * D + j);
        const double u1 = (u_pm1(key, 2 * jj) + 1.0) * 0.5, u2 = (u_pm1(key, 2 * jj + 1) + 1.0) * 0.5;
        return sqrt(-2.0 * log1p(-u1)) * cos(2.0 * 3.141592653589793 * u2);
    };
    auto ggt = [&](int x, int y) {
        double acc = 0.0;
        for (int j = 0; j < D; ++j) acc += g(x, j) * g(y, j);
        return acc;
    };
    if (!t.hb) return ggt(a, b);
    // G G^T is real symmetric: Hermitian-basis coordinates v_aa, (v_ab + v_ba) / sqrt 2 for a < b,
    // 0 for a > b
    if (a == b) return ggt(a, a);
    if (a > b) return 0.0;
    return (ggt(a, b) + ggt(b, a)) / sqrt(2.0);
}
__global__ void k_msg_init(const MsgInitTask* __restrict__ tasks, int ntasks) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntasks) return;
    const MsgInitTask& t = tasks[i];
    double total = 1.0;
    for (int s = 0; s < t.nsites; ++s) {
        const uint64_t key = rng_key(t.seed, t.stream + (uint64_t)s);
        double n2 = 0.0;
        for (int k = 0; k < t.K; ++k) {
            const double v = init_entry(t, key, k);
            n2 += v * v;
            t.dst[s][(long long)k * t.kstride[s] * t.cw] = v;
        }
        total *= sqrt(n2);
    }
    for (int k = 0; k < t.K; ++k) {
        double* p = t.dst[0] + (long long)k * t.kstride[0] * t.cw;
        *p = *p / total;
    }
}
cudaError_t launch_msg_init(const MsgInitTask* d_tasks, int ntasks, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    k_msg_init<<<(ntasks + 63) / 64, 64, 0, s>>>(d_tasks, ntasks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- inner products
// *out = 2^(ea + eb) sum_x A[x] B[x] over n scalars, no conjugation (the last contraction of a
// read-out closing): one CTA per task, four partial sums per thread, the block's sums added
// in a fixed order (the result does not depend on timing).
__device__ __forceinline__ int exp_or_zero(const int* e) { return e ? *e : 0; }
__device__ __forceinline__ double scale2(double v, int e) { return ldexp(v, e); }
__device__ __forceinline__ double2 scale2(double2 v, int e) { return make_double2(ldexp(v.x, e), ldexp(v.y, e)); }
template <typename S>
__global__ void __launch_bounds__(256) k_dot(const DotTask* __restrict__ tasks) {
    const DotTask& t = tasks[blockIdx.x];
    __shared__ S red[32];
    const S* __restrict__ a = (const S*)t.A;
    const S* __restrict__ b = (const S*)t.B;
    S p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = zero<S>();
    long long i = threadIdx.x;
    for (; i + 768 < t.n; i += 1024) {
#pragma unroll
        for (int q = 0; q < 4; ++q) mac(p[q], a[i + 256 * q], b[i + 256 * q]);
    }
    for (; i < t.n; i += 256) mac(p[0], a[i], b[i]);
    const S v = block_sum(add(add(p[0], p[1]), add(p[2], p[3])), red);
    if (threadIdx.x == 0) *(S*)t.out = scale2(v, exp_or_zero(t.ea) + exp_or_zero(t.eb));
}

// Power-of-two normalisation of a buffer of n doubles (2n for complex scalars): the largest
// magnitude is found on the bit patterns (for finite doubles the order of |x| is the integer
// order of the bits without the sign), and the scaling by 2^-e is exact.
__global__ void __launch_bounds__(256) k_pow2norm(const DotTask* __restrict__ tasks, int cplx) {
    const DotTask& t = tasks[blockIdx.x];
    __shared__ unsigned long long red[8];
    double* x = (double*)t.A;
    const long long n = t.n * (cplx ? 2 : 1);
    unsigned long long m = 0;
    for (long long i = threadIdx.x; i < n; i += 256) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull;
        m = u > m ? u : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = red[0];
    for (int w = 1; w < 8; ++w) m = red[w] > m ? red[w] : m;
    int e = 0;
    if (m != 0 && m < 0x7FF0000000000000ull) frexp(__longlong_as_double((long long)m), &e);
    if (e != 0) {
        const double sc = ldexp(1.0, -e);
        for (long long i = threadIdx.x; i < n; i += 256) x[i] *= sc;
    }
    if (threadIdx.x == 0) *(int*)t.out = e + exp_or_zero(t.ea);
}

cudaError_t launch_dot(const DotTask* d_tasks, int ntasks, bool cplx, cudaStream_t s, int normalise) {
    if (ntasks <= 0) return cudaSuccess;
    if (normalise)
        k_pow2norm<<<ntasks, 256, 0, s>>>(d_tasks, cplx ? 1 : 0);
    else if (cplx)
        k_dot<double2><<<ntasks, 256, 0, s>>>(d_tasks);
    else
        k_dot<double><<<ntasks, 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- read-out ratios
// <O> = N_O / N_I in FP64 (App. A read-out), the complex quotient by Smith's algorithm
// (R. L. Smith, CACM 1962: scale by the larger part of the divisor, no intermediate overflow).
__global__ void k_ratio(const RatioTask* __restrict__ tasks, int ntasks, const double* __restrict__ clos, int cplx,
                        double* __restrict__ out, int* status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntasks) return;
    const RatioTask& r = tasks[t];
    auto val = [&](int c) { return cplx ? make_double2(clos[2 * c], clos[2 * c + 1]) : make_double2(clos[c], 0.0); };
    double nr = 0.0, ni = 0.0;
    for (int k = 0; k < r.nparts; ++k) {
        const double2 v = val(r.part[k]);
        nr += r.c_re[k] * v.x - r.c_im[k] * v.y;
        ni += r.c_re[k] * v.y + r.c_im[k] * v.x;
    }
    const double2 d = val(r.denom);
    double qr, qi;
    if (d.x == 0.0 && d.y == 0.0) {
        atomicExch(status, 1);
        qr = qi = 0.0;
    } else if (fabs(d.y) <= fabs(d.x)) {
        const double e = d.y / d.x, f = d.x + d.y * e;
        qr = (nr + ni * e) / f;
        qi = (ni - nr * e) / f;
    } else {
        const double e = d.x / d.y, f = d.y + d.x * e;
        qr = (nr * e + ni) / f;
        qi = (ni * e - nr) / f;
    }
    out[2 * t] = qr;
    out[2 * t + 1] = qi;
}
cudaError_t launch_ratio(const RatioTask* d_tasks, int ntasks, const void* closings, bool cplx, double* out,
                         int* status, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    k_ratio<<<(ntasks + 127) / 128, 128, 0, s>>>(d_tasks, ntasks, (const double*)closings, cplx ? 1 : 0, out, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- dtype conversion
// in_dtype: 0 f64, 1 c128, 2 f32, 3 c64 (the bbp_dtype values).  n = scalar count.
__global__ void k_convert(const void* in, int in_dtype, void* out, long long n, int cplx_out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        switch (in_dtype) {
            case 0: re = ((const double*)in)[i]; break;
            case 1: re = ((const double*)in)[2 * i]; im = ((const double*)in)[2 * i + 1]; break;
            case 2: re = ((const float*)in)[i]; break;
            default: re = ((const float*)in)[2 * i]; im = ((const float*)in)[2 * i + 1]; break;
        }
        if (cplx_out) {
            ((double*)out)[2 * i] = re;
            ((double*)out)[2 * i + 1] = im;
        } else {
            ((double*)out)[i] = re;
        }
    }
}
cudaError_t launch_convert(const void* in, int in_dtype, void* out, long long n, bool cplx_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    k_convert<<<(unsigned)b, 256, 0, s>>>(in, in_dtype, out, n, cplx_out ? 1 : 0);
    return cudaGetLastError();
}

__global__ void k_copy(const uint4* in, uint4* out, long long n16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i];
}
cudaError_t launch_copy(const void* in, void* out, long long bytes, cudaStream_t s) {
    if (bytes <= 0) return cudaSuccess;
    // every buffer in the arena is 256-byte aligned and sized in multiples of 16 bytes
    const long long n16 = bytes / 16;
    long long b = (n16 + 255) / 256;
    if (b > 2048) b = 2048;
    k_copy<<<(unsigned)b, 256, 0, s>>>((const uint4*)in, (uint4*)out, n16);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused column pair (read-out)
template <typename S>
__global__ void k_fuse(const FuseTask* __restrict__ tasks) {
    const FuseTask& t = tasks[blockIdx.y];
    const long long total = (long long)t.u1 * t.u2 * t.l1 * t.d1 * t.d2 * t.r2;
    const S* A = (const S*)t.A;
    const S* B = (const S*)t.B;
    S* out = (S*)t.out;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int r2 = (int)(r % t.r2); r /= t.r2;
        const int d2 = (int)(r % t.d2); r /= t.d2;
        const int d1 = (int)(r % t.d1); r /= t.d1;
        const int l1 = (int)(r % t.l1); r /= t.l1;
        const int u2 = (int)(r % t.u2); r /= t.u2;
        const int u1 = (int)r;
        const S* a = A + u1 * t.a_u + l1 * t.a_l + d1 * t.a_d;
        const S* b = B + u2 * t.b_u + d2 * t.b_d + r2 * t.b_r;
        S acc = zero<S>();
        for (int m = 0; m < t.m; ++m) mac(acc, a[m * t.a_r], b[m * t.b_l]);
        out[e] = acc;
    }
}
cudaError_t launch_fuse(const FuseTask* d_tasks, int ntasks, long long max_out, bool cplx, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    long long bx = (max_out + 255) / 256;
    if (bx > 4096) bx = 4096;
    dim3 grid((unsigned)bx, ntasks);
    if (cplx)
        k_fuse<double2><<<grid, 256, 0, s>>>(d_tasks);
    else
        k_fuse<double><<<grid, 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- typed 4-D relayout
__global__ void k_relayout(const RelayoutTask* __restrict__ tasks) {
    const RelayoutTask& t = tasks[blockIdx.y];
    const long long total = (long long)t.d[0] * t.d[1] * t.d[2] * t.d[3];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int i3 = (int)(r % t.d[3]); r /= t.d[3];
        const int i2 = (int)(r % t.d[2]); r /= t.d[2];
        const int i1 = (int)(r % t.d[1]); r /= t.d[1];
        const int i0 = (int)r;
        const long long so = i0 * t.ss[0] + i1 * t.ss[1] + i2 * t.ss[2] + i3 * t.ss[3];
        const long long dof = i0 * t.ds[0] + i1 * t.ds[1] + i2 * t.ds[2] + i3 * t.ds[3];
        store_split(t.dst, dof, t.dst_kind, load_kind(t.src, so, t.src_kind), t.x3, t.kseg);
    }
}
cudaError_t launch_relayout(const RelayoutTask* d_tasks, int ntasks, long long max_elems, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    long long bx = (max_elems + 255) / 256;
    if (bx > 1024) bx = 1024;
    k_relayout<<<dim3((unsigned)bx, ntasks), 256, 0, s>>>(d_tasks);
    return cudaGetLastError();
}

}  // namespace bbp
