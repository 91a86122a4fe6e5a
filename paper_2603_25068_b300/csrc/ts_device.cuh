// Device-side building blocks shared by the simulator kernels (sm_103a).
//
// Every floating-point operation that can decide an integer (arrival, vacancy,
// link choice, merge) is written with explicit round-to-nearest intrinsics so
// that no multiply-add is contracted: the result is the IEEE single-precision
// value of each operation in the stated order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ts {

constexpr int kTagFree = 0, kTagCong = 1, kTagStop = 2;
constexpr int kTgtNone = -1, kTgtSink = -2, kTgtBlocked = -3;
constexpr int kVehWaiting = -1, kVehArrived = -2;
constexpr unsigned kFull = 0xffffffffu;

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the Philox S-box
// (multipliers 0xD2511F53, 0xCD9E8D57) with Weyl key increments
// 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;   // one wide multiply each
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// Natural logarithm of a positive normal float: x = 2^e m, m in (sqrt(1/2),
// sqrt(2)], log m = 2 atanh((m-1)/(m+1)) by its series through the 11th power,
// e*ln2 added in a 12-bit high part and a low part (Cody & Waite 1980).  Error
// within 2 ulp; every operation rounded to nearest with no contraction.
__device__ __forceinline__ float log32(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float f = __fsub_rn(m, 1.0f);
    const float d = __fadd_rn(m, 1.0f);
    const float r = __fdiv_rn(f, d);
    const float r2 = __fmul_rn(r, r);
    float p = 0x1.745d18p-4f;
    p = __fadd_rn(0x1.c71c72p-4f, __fmul_rn(r2, p));
    p = __fadd_rn(0x1.24924ap-3f, __fmul_rn(r2, p));
    p = __fadd_rn(0x1.99999ap-3f, __fmul_rn(r2, p));
    p = __fadd_rn(0x1.555556p-2f, __fmul_rn(r2, p));
    const float q = __fmul_rn(r2, p);
    const float lm = __fmul_rn(2.0f, __fadd_rn(r, __fmul_rn(r, q)));
    const float fe = (float)e;
    const float hi = __fmul_rn(fe, 0x1.62ep-1f);
    const float lo = __fmul_rn(fe, 0x1.0bfbe8p-15f);
    return __fadd_rn(hi, __fadd_rn(lm, lo));
}

// Gumbel(0,1) for (vehicle, step, stream, slot): word slot&3 of the Philox block
// slot>>2, mapped to U = ((w >> 9) + 1/2) 2^-23 (exact), g = -log(-log U).
__device__ __forceinline__ float gumbel_of_word(uint32_t w) {
    const float u = __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 0x1p-23f);
    return -log32(-log32(u));
}
__device__ __forceinline__ uint4 gumbel_block(uint32_t k0, uint32_t k1, int vid, int t, int stream, int blk) {
    return philox4x32_10(make_uint4((uint32_t)vid, (uint32_t)t, (uint32_t)stream, (uint32_t)blk), k0, k1);
}
__device__ __forceinline__ float gumbel(uint32_t k0, uint32_t k1, int vid, int t, int stream, int slot) {
    const uint4 o = gumbel_block(k0, k1, vid, t, stream, slot >> 2);
    const int s = slot & 3;
    return gumbel_of_word(s == 0 ? o.x : s == 1 ? o.y : s == 2 ? o.z : o.w);
}

// 64-bit merge word: order-preserving image of the float key in the high half,
// ~vehicle id in the low half, so that atomicMax keeps the largest key and, on
// equal keys, the lowest vehicle id.  Zero never occurs for a real entry.
__device__ __forceinline__ unsigned long long merge_word(float key, int vid) {
    const uint32_t b = __float_as_uint(key);
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)o << 32) | (unsigned long long)(~(uint32_t)vid);
}
__device__ __forceinline__ int merge_vid(unsigned long long w) { return (int)(~(uint32_t)(w & 0xffffffffull)); }

// Newell car-following update of one vehicle (SI-A): headway h to the vehicle
// ahead (M for the leader), displacement min(u dt, max(h - s, 0)), TG clip at L.
// Also returns the dead-band tag of the min/max branch used by the adjoint.
__device__ __forceinline__ float newell(float x, float h, float len, float udt, float s, float dtag, int &tag) {
    const float d = __fsub_rn(h, s);
    const float dxc = fmaxf(d, 0.0f);
    const float dx = fminf(udt, dxc);
    const float xp = __fadd_rn(x, dx);
    tag = (d <= dtag) ? kTagStop : (d >= __fsub_rn(udt, dtag) ? kTagFree : kTagCong);
    return fminf(xp, len);
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

}  // namespace ts
