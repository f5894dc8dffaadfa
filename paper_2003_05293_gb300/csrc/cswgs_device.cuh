// Device primitives of the CS-WGS kernels: the seeded draws (theta^0 and the
// per-iteration pixel subsets), the fixed-point lens-and-prism phase of Eq. 2
// with its exact range reduction, and sincos of a fixed-point phase.
#pragma once

#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

namespace cswgs {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318530717958647692f;

// ------------------------------------------------------------ seeded draws --
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), counter form: output k of the
// sequence whose state starts at `seed` and advances by the golden gamma.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// MurmurHash3 32-bit finaliser (Appleby).
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// theta_n^0 in turns, as a 53-bit fraction of [0, 1): the random phases of
// the random-superposition start (Eq. 1).  Draw n of the seed's sequence.
__host__ __device__ __forceinline__ double theta0_turns(uint64_t seed, int n)
{
    return (double)(splitmix64(seed, (uint64_t)n) >> 11) * 0x1.0p-53;
}

// Round keys of the subset permutation of iteration j: outputs 2^32 + 4j + r
// of the seed's sequence, upper 32 bits.
struct SubsetKeys {
    uint32_t k0, k1, k2, k3;
};

__host__ __device__ __forceinline__ SubsetKeys subset_keys(uint64_t seed, int j)
{
    uint64_t base = 0x100000000ull + 4ull * (uint64_t)(uint32_t)j;
    SubsetKeys K;
    K.k0 = (uint32_t)(splitmix64(seed, base + 0) >> 32);
    K.k1 = (uint32_t)(splitmix64(seed, base + 1) >> 32);
    K.k2 = (uint32_t)(splitmix64(seed, base + 2) >> 32);
    K.k3 = (uint32_t)(splitmix64(seed, base + 3) >> 32);
    return K;
}

// One round (L, R) -> (R, (L + F(R)) mod p), F(R) = floor(fmix32(R ^ key) p / 2^32),
// p the modulus of the incoming L.
__device__ __forceinline__ void feistel_round(uint32_t &L, uint32_t &R, uint32_t key, uint32_t p)
{
    uint32_t F = __umulhi(fmix32(R ^ key), p);   // in [0, p)
    uint32_t nr = L + F;
    nr = nr >= p ? nr - p : nr;                  // (L + F) mod p, both < p
    L = R;
    R = nr;
}

// Exact division by a divisor d fixed for many dividends: with the reciprocal
// m = floor((2^32 - 1) / d), umulhi(x, m) is floor(x / d) or one less for
// every 32-bit x (the product undershoots x / d by less than x / 2^32 < 1), and
// one comparison of the remainder settles it.
struct UDiv {
    uint32_t d, m;
};

__host__ __device__ __forceinline__ UDiv udiv_of(uint32_t d) { return UDiv{d, 0xFFFFFFFFu / d}; }

__device__ __forceinline__ uint32_t udiv(uint32_t x, const UDiv &v, uint32_t &r)
{
    uint32_t q = __umulhi(x, v.m);
    r = x - q * v.d;
    if (r >= v.d) {
        ++q;
        r -= v.d;
    }
    return q;
}

// Keyed bijection of [0, a b): k = L b + R with L in [0, a), R in [0, b);
// four rounds whose moduli alternate a, b, a, b (each round swaps the two
// halves' ranges); result L b + R.
__device__ __forceinline__ uint32_t permute_rect(uint32_t k, uint32_t a, const UDiv &b, const SubsetKeys &K)
{
    uint32_t R;
    uint32_t L = udiv(k, b, R);
    feistel_round(L, R, K.k0, a);
    feistel_round(L, R, K.k1, b.d);
    feistel_round(L, R, K.k2, a);
    feistel_round(L, R, K.k3, b.d);
    return L * b.d + R;
}

__device__ __forceinline__ uint32_t permute_rect(uint32_t k, uint32_t a, uint32_t b, const SubsetKeys &K)
{
    return permute_rect(k, a, udiv_of(b), K);
}

// pi_{seed,j}(k): keyed bijection of [0, P^2), the square grid's subset order.
// The subset S_j of an iteration is the image of [0, Mp) (Section 2, CS-WGS;
// Section 3, "Compressed sensing": a random pixel order, c M pixels per
// iteration).
__device__ __forceinline__ uint32_t permute(uint32_t k, uint32_t P, const SubsetKeys &K)
{
    return permute_rect(k, P, P, K);
}

// Keyed bijection of [0, D) for any D, on the rectangle a x b >= D (a the
// smallest integer with a^2 >= D, b = ceil(D / a)): values that land at or
// beyond D go through the rectangle's permutation again (cycle walking).  The
// walk from k < D meets at most a b - D values >= D before it returns below
// D, so the loop bound never cuts a walk short; the final clamp only keeps a
// corrupted input in range.
__device__ __forceinline__ uint32_t permute_domain(uint32_t k, uint32_t D, uint32_t a, const UDiv &b,
                                                   const SubsetKeys &K)
{
    uint32_t y = permute_rect(k, a, b, K);
    const uint32_t extra = a * b.d - D;
    for (uint32_t s = 0; y >= D && s < extra; ++s) y = permute_rect(y, a, b, K);
    return y < D ? y : 0u;
}

// Host side: the rectangle of permute_domain for a domain of D >= 1 values.
inline void permute_rect_of(uint32_t D, uint32_t *a, uint32_t *b)
{
    uint64_t x = (uint64_t)sqrt((double)D);
    while (x * x < D) ++x;
    while (x > 1 && (x - 1) * (x - 1) >= D) --x;
    if (x == 0) x = 1;
    *a = (uint32_t)x;
    *b = (uint32_t)((D + x - 1) / x);
}

// ------------------------------------------------------ fixed-point phase --
// Phases are carried in turns as 32-bit fixed point (2^32 = one turn), so
// arithmetic mod 2^32 is arithmetic mod 2 pi with no rounding: the range
// reduction of the lens-and-prism argument (Eq. 2, up to a few hundred turns
// at P = 1152) is exact.  The spot coefficients (turns per pixel, FP64 in the
// preparation kernel) are split into 32-bit words:
//   tilt:    A = a * 2^32, B = b * 2^32           (a = alpha/P, b = beta/P)
//   defocus: g * 2^32 = Gh + Gl * 2^-32            (g = gamma/(P/2)^2)
// so that, for integer pixel coordinates x', y' and rho^2 = x'^2 + y'^2 < 2^32,
//   phi_n(m) * 2^32 / (2 pi) = A x' + B y' + Gh rho^2 + Gl rho^2 2^-32   (mod 2^32).
// The first three terms are exact integer arithmetic.  The last one is below
// rho^2 units (< 2^-12 turn, 1.5e-3 rad at P = 1152), so it is carried in
// floating point, in radians (gl = Gl 2^-64 2 pi per unit of rho^2), and
// added after the conversion to radians with an absolute error ~1e-10 rad.
struct SpotFix {
    int32_t A, B, Gh;
    float gl;       // radians per unit of rho^2 (the low word of the defocus)
};

// Nearest 32-bit fixed-point turn of a real number of turns (mod 1).
__device__ __forceinline__ uint32_t turns_to_fix(double t)
{
    double f = t - rint(t);                        // [-0.5, 0.5], exact
    return (uint32_t)(int64_t)llrint(f * 4294967296.0);
}

__device__ __forceinline__ SpotFix spot_fix(double alpha, double beta, double gamma, int P)
{
    SpotFix s;
    s.A = (int32_t)turns_to_fix(alpha / (double)P);
    s.B = (int32_t)turns_to_fix(beta / (double)P);
    double half = 0.5 * (double)P;
    double g = gamma / (half * half);
    g = g - rint(g);                               // rho^2 is an integer: g mod 1
    double gs = g * 4294967296.0;                  // exact scaling
    double gh = floor(gs);
    double frac = gs - gh;                         // [0, 1) units of 2^-32 turn per rho^2
    s.Gh = (int32_t)(uint32_t)(int64_t)gh;
    s.gl = (float)(frac * (kTwoPi / 4294967296.0));
    return s;
}

// Integer part of the fixed-point phase of spot s at pixel (x', y', rho^2),
// plus an addend.
__device__ __forceinline__ uint32_t fix_phase(const SpotFix &s, int32_t xp, int32_t yp,
                                              uint32_t rho2, uint32_t addend)
{
    uint32_t t = addend + (uint32_t)s.A * (uint32_t)xp;
    t += (uint32_t)s.B * (uint32_t)yp;
    t += (uint32_t)s.Gh * rho2;
    return t;
}

// Rounding bias folded into every addend: the conversion below keeps the top
// 23 bits of the phase, so adding half of the dropped range rounds to nearest.
constexpr uint32_t kFixRound = 1u << 8;

// sin and cos of 2 pi T / 2^32 + corr, T already carrying kFixRound, where
// corr_m2pi = corr - 2 pi.  The top 23 bits of T become the mantissa of a float
// in [1, 2), i.e. 1 + turns; one FMA turns it into radians in [0, 2 pi) plus
// the small correction; the hardware sine/cosine approximations finish.
__device__ __forceinline__ void sincos_fix(uint32_t T, float corr_m2pi, float &s, float &c)
{
    float f = __uint_as_float((T >> 9) | 0x3F800000u);
    float x = fmaf(f, kTwoPiF, corr_m2pi);
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// ------------------------------------------------ half-precision sincos --
// Option for the compressed iterations: sine and cosine of two fixed-point
// phases at once in packed FP16 arithmetic on the FMA pipe (no SFU).  T1, T2
// carry kHalfAddend (half a turn, so the value below is centred on 0, plus
// the rounding of the top 10 bits).  Their top 10 bits become the mantissas
// of a half2 in [1, 2); t = f - 1.5 is the turn in [-1/2, 1/2).  With the
// half angle pi t in [-pi/2, pi/2]:
//   s = sqrt2 sin(pi t) ~ t (S1 + S3 t^2 + S5 t^4),
//   c = sqrt2 cos(pi t) ~ C0 + C2 t^2 + C4 t^4,
//   sin(2 pi t) = s c,  cos(2 pi t) = c^2 - 1.
// Coefficients: a minimax-weighted least-squares fit of sin(pi t), cos(pi t)
// on [-1/2, 1/2], times sqrt 2, rounded to FP16, then moved by a few FP16
// steps so that the evaluated phasors (in FP16 arithmetic, on the 1024 inputs
// the 10-bit phase can take) average to zero within 1e-5.  A non-zero mean
// adds the same complex offset to every projected spot field and biases the
// spot phases; the rest of the error is noise that averages out over pixels.
// Error against the exact phase: 1.2e-3 rad RMS, |phasor - exact| <= 4.6e-3.
constexpr uint32_t kHalfAddend = (1u << 31) + (1u << 21);

__device__ __forceinline__ __half2 half2_bits(unsigned short bits)
{
    __half2_raw r;
    r.x = bits;
    r.y = bits;
    return __half2(r);
}

__device__ __forceinline__ void sincos_fix_h2(uint32_t T1, uint32_t T2, __half2 &s, __half2 &c)
{
    const uint32_t p = __byte_perm(T1, T2, 0x7632);              // top 16 bits of each
    const uint32_t h = ((p >> 6) & 0x03FF03FFu) | 0x3C003C00u;   // 1 + top 10 bits / 1024
    const __half2 t = __hsub2(*reinterpret_cast<const __half2 *>(&h), half2_bits(0x3E00));   // - 1.5
    const __half2 z = __hmul2(t, t);
    __half2 ps = __hfma2(z, half2_bits(0x4281), half2_bits(0xC746));   // S5 = 3.2519, S3 = -7.2734
    ps = __hfma2(z, ps, half2_bits(0x4472));                            // S1 = 4.4453
    ps = __hmul2(ps, t);
    __half2 pc = __hfma2(z, half2_bits(0x450E), half2_bits(0xC6E9));   // C4 = 5.0547, C2 = -6.9102
    pc = __hfma2(z, pc, half2_bits(0x3DA7));                            // C0 = 1.4131
    s = __hmul2(ps, pc);
    c = __hfma2(pc, pc, half2_bits(0xBC00));                            // - 1
}

// Fixed-point turn of an angle in radians, as float (|x| <= pi).
__device__ __forceinline__ uint32_t rad_to_fix(float x)
{
    // 2^32 / (2 pi) = 683565275.58...
    return (uint32_t)__float2int_rn(x * 683565275.5764316f);
}

}  // namespace cswgs
