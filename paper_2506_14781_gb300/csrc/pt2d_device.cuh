// Device arithmetic of the 2D-PT library: counter-based random words, the
// project's single-precision exponential, the heat-bath decision and the swap
// test.  Every sequence here is the library's numerical contract (stated in
// include/pt2d.h); the CPU oracle implements the same contract independently.
#pragma once

#include <cstdint>

namespace pt2d {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2,
//   x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0),
// with the key advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;  // 2^32 * (golden ratio - 1)
constexpr uint32_t kWeyl1 = 0xBB67AE85u;  // 2^32 * (sqrt(3) - 1)

enum : uint32_t { kTagInit = 0u, kTagSweep = 1u, kTagSwap = 2u };

// One Philox4x32 round with round key (k0, k1).
__device__ __forceinline__ uint4 philox_round(uint4 x, uint32_t k0, uint32_t k1) {
    const uint32_t lo0 = kPhiloxM0 * x.x;
    const uint32_t hi0 = __umulhi(kPhiloxM0, x.x);
    const uint32_t lo1 = kPhiloxM1 * x.z;
    const uint32_t hi1 = __umulhi(kPhiloxM1, x.z);
    return make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        x = philox_round(x, k0, k1);
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    return x;
}

// The ten round keys of one seed, precomputed on the host and passed as a
// kernel parameter so the key schedule costs no per-thread instructions.
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline RoundKeys round_keys(uint64_t seed) {
    RoundKeys rk;
    uint32_t a = static_cast<uint32_t>(seed), b = static_cast<uint32_t>(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        rk.k0[i] = a;
        rk.k1[i] = b;
        a += kWeyl0;
        b += kWeyl1;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, const RoundKeys &rk) {
#pragma unroll
    for (int round = 0; round < 10; ++round) x = philox_round(x, rk.k0[round], rk.k1[round]);
    return x;
}

// Uniform on the 2^23-point grid of (0, 1]: u = ((r >> 9) + 1) * 2^-23, exactly.
__device__ __forceinline__ float uniform23(uint32_t r) {
    return __fmul_rn(__uint2float_rn((r >> 9) + 1u), 0x1p-23f);
}

// ---------------------------------------------------------------------------
// pt_exp: e^x by additive range reduction x = k ln2 + r with ln 2 split into
// a float whose low 12 significand bits are zero (so k * LN2_HI is exact) and
// the rounded remainder, then the Taylor polynomial sum_{n<=7} r^n / n! in
// Horner form, then scaling by 2^k through the exponent field in two steps
// where 2^k alone would leave the normal range.  Each operation rounds to
// nearest on its own (no contraction).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pow2i(int m) {  // 2^m, -126 <= m <= 127
    return __uint_as_float(static_cast<uint32_t>(m + 127) << 23);
}

static __device__ __noinline__ float pt_exp(float x) {
    const float kL2E = 0x1.715476p+0f;     // RN(log2 e)
    const float kLn2Hi = 0x1.62ep-1f;      // RN(ln 2) with 12 low bits cleared
    const float kLn2Lo = 0x1.0bfbe8p-15f;  // RN(ln 2 - kLn2Hi)
    const float kC7 = 0x1.a01a02p-13f;     // RN(1/7!)
    const float kC6 = 0x1.6c16c2p-10f;     // RN(1/6!)
    const float kC5 = 0x1.111112p-7f;      // RN(1/5!)
    const float kC4 = 0x1.555556p-5f;      // RN(1/4!)
    const float kC3 = 0x1.555556p-3f;      // RN(1/3!)
    const float kC2 = 0x1p-1f;
    const float kC1 = 0x1p+0f;
    const float kC0 = 0x1p+0f;
    if (x != x) return x;
    if (x > 88.75f) return __int_as_float(0x7f800000);
    if (x < -104.0f) return 0.0f;
    const float kf = rintf(__fmul_rn(x, kL2E));
    const int k = static_cast<int>(kf);
    const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, kLn2Hi)), __fmul_rn(kf, kLn2Lo));
    float p = kC7;
    p = __fadd_rn(__fmul_rn(p, r), kC6);
    p = __fadd_rn(__fmul_rn(p, r), kC5);
    p = __fadd_rn(__fmul_rn(p, r), kC4);
    p = __fadd_rn(__fmul_rn(p, r), kC3);
    p = __fadd_rn(__fmul_rn(p, r), kC2);
    p = __fadd_rn(__fmul_rn(p, r), kC1);
    p = __fadd_rn(__fmul_rn(p, r), kC0);
    if (k > 127) return __fmul_rn(__fmul_rn(p, pow2i(k - 64)), pow2i(64));
    if (k < -126) return __fmul_rn(__fmul_rn(p, pow2i(k + 64)), pow2i(-64));
    return __fmul_rn(p, pow2i(k));
}

// ---------------------------------------------------------------------------
// Heat-bath decision, exact contract: t = beta*float(H); e = pt_exp(-t);
// d = 1 + e; v = u*d; +1 iff v < 1.
// ---------------------------------------------------------------------------
static __device__ __noinline__ int heatbath_exact(float beta, int32_t H, uint32_t r) {
    const float t = __fmul_rn(beta, __int2float_rn(H));
    const float e = pt_exp(-t);
    const float d = __fadd_rn(1.0f, e);
    const float v = __fmul_rn(uniform23(r), d);
    return v < 1.0f ? 1 : -1;
}

// Fast path.  e~ = 2^y with y = (-beta log2 e) * H from the hardware
// approximation, d~ = 1 + e~ and t~ = u d~ - 1 (one fused multiply-add).  Near
// the decision boundary (t ~ 0, so |y| <= 24) the contract's v = u (x) d and
// 1 + t~ differ by at most ~2^-17.5 relative (argument rounding on both sides,
// pt_exp's <= 3 ulp, ex2.approx's ~2^-22), so outside the band |t~| <= 2^-14
// the sign of t~ is the contract's answer (t~ < 0 <=> +1); inside the band the
// exact contract decides.  u > 0, so an infinite e~ gives t~ = +inf (-1), as
// the contract's v = u * inf does.
__device__ __forceinline__ float ex2_approx(float y) {
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
    return e;
}

constexpr float kBand = 0x1p-14f;

// t~ of the fast path (see above); nbl2e = -beta * log2(e), rounded once per walker.
__device__ __forceinline__ float heatbath_fast(float nbl2e, int32_t H, uint32_t r) {
    const float e = ex2_approx(nbl2e * __int2float_rn(H));
    const float u = __uint_as_float(0x3f800001u + (r >> 9)) - 1.0f;  // ((r >> 9) + 1) * 2^-23
    return fmaf(u, 1.0f + e, -1.0f);
}

// Returns a float whose sign is the decision: negative <=> new spin +1.
__device__ __forceinline__ float heatbath_t(float beta, float nbl2e, int32_t H, uint32_t r) {
    const float t = heatbath_fast(nbl2e, H, r);
    if (fabsf(t) > kBand) return t;
    return heatbath_exact(beta, H, r) > 0 ? -1.0f : 1.0f;
}

__device__ __forceinline__ int heatbath(float beta, float nbl2e, int32_t H, uint32_t r) {
    return heatbath_t(beta, nbl2e, H, r) < 0.0f ? 1 : -1;
}

// Metropolis swap test: accept iff x >= 0 or u <= pt_exp(x).
__device__ __forceinline__ bool swap_accept(float x, uint32_t r) {
    if (x >= 0.0f) return true;
    return uniform23(r) <= pt_exp(x);
}

}  // namespace pt2d
