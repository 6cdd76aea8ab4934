// rt_device.cuh -- device-side building blocks of the shortwave Monte Carlo
// tracer (Veerman et al. 2022, Sec. 2.3): counter-based random numbers, the
// phase-function samplers, the direction update and the Lambertian surface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rt {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32
// multiplies with a Weyl-sequence key schedule. Keyed by the 64-bit seed; the
// counter is (photon id lo, photon id hi, block index, slot), so the stream of
// a photon does not depend on which thread or launch traces it.
// ---------------------------------------------------------------------------
struct Philox {
    static constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    static constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
};

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(Philox::M0, c.x), lo0 = Philox::M0 * c.x;
        const uint32_t hi1 = __umulhi(Philox::M1, c.z), lo1 = Philox::M1 * c.z;
#else
        const uint64_t p0 = (uint64_t)Philox::M0 * c.x, p1 = (uint64_t)Philox::M1 * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += Philox::W0;
        k1 += Philox::W1;
    }
    return c;
}

// Uniform float in the open interval (0,1) from the top 23 bits m of a word:
// the float 1 + m 2^-23 (those bits as its mantissa) minus 1 - 2^-24 is
// exactly (m + 1/2) 2^-23, so -log(u) is always finite. Integer and add
// instructions only, no int-to-float conversion.
__device__ __forceinline__ float u01_bits23(uint32_t m)
{
    return __uint_as_float(0x3F800000u | m) - 0.99999994039535522461f;
}

__device__ __forceinline__ float u01(uint32_t x) { return u01_bits23(x >> 9); }

// A fifth uniform from one Philox block: the low 9 bits of words 0 and 1 and
// the low 5 of word 2 (23 bits), which u01 discards. The bits of a uniformly
// random word are independent, so this is independent of the four uniforms
// taken from the top bits.
__device__ __forceinline__ float u01_low(uint4 r)
{
    return u01_bits23((r.x & 0x1FFu) | ((r.y & 0x1FFu) << 9) | ((r.z & 0x1Fu) << 18));
}

// (float)i for |i| < 2^22 with an integer add and a float subtract (no
// conversion instruction): i added to the bits of 1.5 * 2^23 gives the float
// 1.5 * 2^23 + i exactly, since floats of that binade are spaced by 1.
__device__ __forceinline__ float small_int_to_float(int i)
{
    return __int_as_float(0x4B400000 + i) - 12582912.0f;
}

// sqrt(x) for x >= 0 from the reciprocal square root (a few units in the last
// place; 0 maps to 0): shorter than the correctly rounded square root.
__device__ __forceinline__ float sqrt_fast(float x)
{
    return x * rsqrtf(fmaxf(x, 1e-30f));
}

// ---------------------------------------------------------------------------
// Sobol start positions (Sec. 2.3: photons enter the domain top at the points
// of a scrambled Sobol sequence). The first two Sobol dimensions in natural
// order, as 32-bit binary fractions: dimension 1 is the base-2 radical inverse
// of k (bit reversal); dimension 2 XORs the direction numbers V_i of the
// primitive polynomial x + 1 (m_1 = 1), V_1 = 2^31 and V_i = V_(i-1) ^
// (V_(i-1) >> 1), over the set bits of k. Each aligned block of 2^m points is a
// (0,m,2)-net; XOR with a fixed random word per axis (a random digital shift)
// keeps that property and makes each point uniform.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t sobol_dim1(uint32_t k)
{
#ifdef __CUDA_ARCH__
    return __brev(k);
#else
    uint32_t r = 0;
    for (int b = 0; b < 32; ++b) r |= ((k >> b) & 1u) << (31 - b);
    return r;
#endif
}

__host__ __device__ __forceinline__ uint32_t sobol_dim2(uint32_t k)
{
    uint32_t v = 0x80000000u, r = 0u;
    for (; k; k >>= 1, v ^= v >> 1)
        if (k & 1u) r ^= v;
    return r;
}

// ---------------------------------------------------------------------------
// Phase functions (Sec. 2.3): Rayleigh for gas, Henyey-Greenstein without
// delta-scaling for cloud droplets. Both by exact inversion of the CDF.
// ---------------------------------------------------------------------------

// Rayleigh p(mu) = 3/8 (1 + mu^2): the CDF (mu^3 + 3 mu + 4)/8 = xi is the
// depressed cubic mu^3 + 3 mu = 2a with a = 4 xi - 2, whose single real root is
// c - 1/c with c = (a + sqrt(a^2 + 1))^(1/3). The root is odd in a, so it is
// evaluated for |a| to avoid cancellation. The base lies in [1, 2 + sqrt 5],
// where the fast power __powf is accurate to a few units in the last place.
__device__ __forceinline__ float rayleigh_mu(float xi)
{
    const float a = 4.0f * xi - 2.0f;
    const float t = fabsf(a);
    const float c = __powf(t + sqrt_fast(fmaf(t, t, 1.0f)), 0.333333343f);
    return copysignf(c - __fdividef(1.0f, c), a);
}

// Henyey-Greenstein: with s = 2 xi - 1 the inverse CDF
//   mu = (1 + g^2 - ((1 - g^2)/(1 + g s))^2) / (2 g)
// expands to a form without the 1/g cancellation, exact at g = 0 (isotropic):
//   mu = (s + g (3 + s^2)/2 + g^2 s + g^3 (s^2 - 1)/2) / (1 + g s)^2.
__device__ __forceinline__ float hg_mu(float g, float xi)
{
    const float s = fmaf(2.0f, xi, -1.0f);
    const float s2 = s * s;
    const float num = s + g * (0.5f * (3.0f + s2) + g * (s + 0.5f * g * (s2 - 1.0f)));
    const float d = fmaf(g, s, 1.0f);
    const float mu = __fdividef(num, d * d);
    return fminf(1.0f, fmaxf(-1.0f, mu));
}

// Azimuth phi = pi (2 xi - 1), uniform on (-pi, pi): (sin phi, cos phi).
__device__ __forceinline__ void azimuth(float xi, float &sp, float &cp)
{
    __sincosf(3.14159265358979f * fmaf(2.0f, xi, -1.0f), &sp, &cp);
}

// Rotate the unit vector u by polar cosine mu and azimuth phi (given as sin,
// cos) about itself, using the frame e1 = (ux uz, uy uz, -(1-uz^2))/sqrt(1-uz^2),
// e2 = (-uy, ux, 0)/sqrt(1-uz^2); renormalised against FP32 drift.
__device__ __forceinline__ void turn(float &ux, float &uy, float &uz, float mu, float sp, float cp)
{
    const float st = sqrt_fast(fmaxf(0.0f, 1.0f - mu * mu));
    float nx, ny, nz;
    const float q = 1.0f - uz * uz;
    if (q > 1e-10f) {
        const float rq = rsqrtf(q);
        const float sq = q * rq;
        nx = st * (ux * uz * cp - uy * sp) * rq + ux * mu;
        ny = st * (uy * uz * cp + ux * sp) * rq + uy * mu;
        nz = -st * cp * sq + uz * mu;
    } else {
        nx = st * cp;
        ny = st * sp;
        nz = uz > 0.0f ? mu : -mu;
    }
    const float rn = rsqrtf(nx * nx + ny * ny + nz * nz);
    ux = nx * rn;
    uy = ny * rn;
    uz = nz * rn;
}

// Lambertian (cosine-law) reflection into the upper hemisphere (Sec. 2.3).
__device__ __forceinline__ void lambert_up(float &ux, float &uy, float &uz, float xi_mu, float xi_phi)
{
    const float mu = sqrt_fast(xi_mu);
    const float st = sqrt_fast(fmaxf(0.0f, 1.0f - xi_mu));
    float sp, cp;
    azimuth(xi_phi, sp, cp);
    ux = st * cp;
    uy = st * sp;
    uz = mu;
}

}  // namespace rt
