// tts_philox.cuh -- counter-based noise for the spin bath.
//
// Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw ("Parallel random
// numbers: as easy as 1, 2, 3", SC'11): a 4-word counter and 2-word key, ten
// rounds, each multiplying words 0 and 2 by the Philox constants, swapping the
// halves of the products into the counter and mixing in the key, with the key
// bumped by the Weyl increments after every round.  Usable on host (alloy
// placement) and device (thermal noise).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define TTS_HD __host__ __device__ __forceinline__
#else
#define TTS_HD inline
#endif

namespace tts {

struct u32x4 {
    uint32_t x, y, z, w;
};

TTS_HD void mul_hi_lo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
    // one widening multiply gives both halves
    const uint64_t p = static_cast<uint64_t>(a) * static_cast<uint64_t>(b);
    hi = static_cast<uint32_t>(p >> 32);
    lo = static_cast<uint32_t>(p);
}

// Division of n < 2^31 by an invariant d >= 1 with one multiply-high, add and
// shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (mulhi(m, n) + n) >> l.
struct FastDiv {
    uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    f.l = 0;
    while ((1ull << f.l) < d) ++f.l;
    f.m = static_cast<uint32_t>(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
    return f;
}

TTS_HD uint32_t fast_div(uint32_t n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = static_cast<uint32_t>((static_cast<uint64_t>(f.m) * n) >> 32);
#endif
    return (t + n) >> f.l;
}

TTS_HD u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t kMulA = 0xD2511F53u;
    constexpr uint32_t kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u;
    constexpr uint32_t kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hA, lA, hB, lB;
        mul_hi_lo(kMulA, c.x, hA, lA);
        mul_hi_lo(kMulB, c.z, hB, lB);
        u32x4 n;
        n.x = hB ^ c.y ^ k0;
        n.y = lB;
        n.z = hA ^ c.w ^ k1;
        n.w = lA;
        c = n;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// The ten round keys (k0 + r W_A, k1 + r W_B), r = 0..9, of a key pair: a
// kernel that receives them as launch parameters XORs constants instead of
// advancing the key in every round.
struct PhiloxRoundKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1)
{
    PhiloxRoundKeys K;
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0;
        K.k1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

TTS_HD u32x4 philox4x32_10(u32x4 c, const PhiloxRoundKeys &K)
{
    constexpr uint32_t kMulA = 0xD2511F53u;
    constexpr uint32_t kMulB = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hA, lA, hB, lB;
        mul_hi_lo(kMulA, c.x, hA, lA);
        mul_hi_lo(kMulB, c.z, hB, lB);
        c = u32x4{hB ^ c.y ^ K.k0[r], lB, hA ^ c.w ^ K.k1[r], lA};
    }
    return c;
}

// Uniform on (0, 1): the top 23 bits plus one half-bit, (2k + 1) * 2^-24, an
// exact float as well as an exact double.
TTS_HD float uniform_f(uint32_t x)
{
    return static_cast<float>((x >> 9) | 0u) * 1.1920928955078125e-07f + 5.9604644775390625e-08f;
}
TTS_HD double uniform_d(uint32_t x)
{
    return static_cast<double>(x >> 9) * 1.1920928955078125e-07 + 5.9604644775390625e-08;
}

// Reserved counter word 2 values of non-thermal streams.
constexpr uint32_t kStreamPlacement = 0xFFFF0000u;

}  // namespace tts
