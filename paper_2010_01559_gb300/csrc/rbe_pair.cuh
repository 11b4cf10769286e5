// rbe_pair.cuh -- the real-space pair terms of the mixed path (Eq. force,
// second term, truncated at r_c; Eq. Ljpotential with r_off = 0), shared by the
// real-space kernels (rbe_real.cu) and the fused structure-factor + list-pass
// launch (rbe_fourier.cu).
#pragma once

#include "rbe_internal.cuh"

namespace rbe {

constexpr int kPartFourier = 1, kPartReal = 2, kPartLJ = 4;

// Deterministic block sum of two doubles (fixed shuffle tree, then warps in
// order); the result is valid in thread 0.
__device__ __forceinline__ double2 block_sum2_real(double a, double b) {
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) { r.x += sa[k]; r.y += sb[k]; }
    }
    return r;
}

struct PairAcc {
    float fx, fy, fz, phr, ec, elj, wc, wlj;     // wc, wlj: half the pair virials r.F
};

// erfc(x) for x >= 0 given e = exp(-x^2): the rational approximation of
// Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26
// (after Hastings), |error| <= 1.5e-7.  It reuses the Gaussian the force needs
// anyway, so erfc costs one reciprocal and five FMAs.
__device__ __forceinline__ float erfc_as(float e, float x) {
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float p = 1.061405429f;
    p = fmaf(p, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    return p * t * e;
}

// Per-system constants of the pair terms, in registers.
struct PairConst {
    float rc2, lj_rc2, alpha, sa, two_sa_spi, lB, lj_s2, lj_eps, lj_shift;
    bool vir;                                   // accumulate the virials
};

// Pair terms for displacement r_ij = (dx, dy, dz), |r_ij|^2 = r2 > 0.
__device__ __forceinline__ void pair_terms(float dx, float dy, float dz, float r2, float qj,
                                           float lbqi, const PairConst& k, PairAcc& acc) {
    const float inv_r = rsqrtf(r2);
    if (r2 < k.rc2) {
        const float x = k.sa * (r2 * inv_r);
        const float ex = __expf(-k.alpha * r2);                  // exp(-x^2)
        const float pot = erfc_as(ex, x) * inv_r;                 // erfc(sqrt(a) r) / r
        const float g_over_r = fmaf(k.two_sa_spi, ex, pot) * inv_r * inv_r;   // G(r) / r
        const float s_ = -lbqi * qj * g_over_r;
        acc.fx = fmaf(s_, dx, acc.fx);
        acc.fy = fmaf(s_, dy, acc.fy);
        acc.fz = fmaf(s_, dz, acc.fz);
        acc.phr = fmaf(k.lB * qj, pot, acc.phr);
        acc.ec = fmaf(0.5f * lbqi * qj, pot, acc.ec);
        // r.F of the pair: lB q_i q_j (erfc(sqrt(a) r)/r + 2 sqrt(a/pi) e^{-a r^2})
        if (k.vir) acc.wc = fmaf(0.5f * lbqi * qj, fmaf(k.two_sa_spi, ex, pot), acc.wc);
    }
    if (r2 < k.lj_rc2) {
        const float inv_r2 = inv_r * inv_r;
        const float sr2 = k.lj_s2 * inv_r2;
        const float sr6 = sr2 * sr2 * sr2;
        const float mag = 24.f * k.lj_eps * (2.f * sr6 * sr6 - sr6) * inv_r2;
        acc.fx = fmaf(-mag, dx, acc.fx);
        acc.fy = fmaf(-mag, dy, acc.fy);
        acc.fz = fmaf(-mag, dz, acc.fz);
        acc.elj += 0.5f * (4.f * k.lj_eps * (sr6 * sr6 - sr6) + k.lj_shift);
        if (k.vir) acc.wlj = fmaf(0.5f * mag, r2, acc.wlj);   // r.F = 24 eps (2 (s/r)^12 - (s/r)^6)
    }
}

// Pair terms from two fixed-point records: the displacement is the 32-bit
// difference of the coordinates, which is the minimum image (|r_ij| < L / 2),
// rounded once to FP32 and scaled to length units.  A zero displacement (the
// particle itself) adds nothing.
__device__ __forceinline__ void pair_fixed(const uint4& si, const uint4& sj, float Lu,
                                           float lbqi, const PairConst& kc, PairAcc& acc) {
    const float dx = (float)(int32_t)(sj.x - si.x) * Lu;
    const float dy = (float)(int32_t)(sj.y - si.y) * Lu;
    const float dz = (float)(int32_t)(sj.z - si.z) * Lu;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 > 0.f) pair_terms(dx, dy, dz, r2, __uint_as_float(sj.w), lbqi, kc, acc);
}

}  // namespace rbe
