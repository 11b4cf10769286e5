// rbe_real.cu -- real-space Coulomb (Eq. force, second term, truncated at r_c),
// shifted Lennard-Jones (Eq. Ljpotential with r_off = 0), the assembly of the
// total force / dE/dq, the Langevin update of Sec. 3.3, and the FP64 energy
// reduction.
//
// G threads per particle (G = 1 .. 32, a tuning choice) in cell order walk the
// 27 cells around the particle's own (cells have side >= r_c, at least 3 per
// edge, so every pair within r_c is met exactly once, as the minimum image).
// Neighbouring particles share most neighbour records, so they are served
// from L1.
//
// Real-space pair terms for r < r_c (r_ij = r_j - r_i):
//   F_i   += -lB q_i q_j G(r) r_ij / r,  G = erfc(sqrt(a) r)/r^2 + 2 sqrt(a) e^{-a r^2}/(sqrt(pi) r)
//   phi_i += lB q_j erfc(sqrt(a) r) / r
//   e_i   += lB q_i q_j erfc(sqrt(a) r) / (2 r)
// LJ for r < R_c: F_i -= 24 eps (2 (s/r)^12 - (s/r)^6) r_ij / r^2,
//   e_i += (4 eps ((s/r)^12 - (s/r)^6) + V_shift) / 2.
//
// Langevin (kick, exact Ornstein-Uhlenbeck, drift; m dv = (F - gamma v) dt +
// sqrt(2 gamma kT) dW): v += (dt/m) F; v = c1 v + c2 xi; r = wrap(r + dt v),
// c1 = exp(-gamma dt / m), c2 = sqrt((1 - c1^2) kT / m), xi from Philox with
// counter (i, 0, step_lo, (stream << 8) | 2) by Box-Muller.
#include <cmath>

#include "rbe_internal.cuh"

namespace rbe {

constexpr int kPartFourier = 1, kPartReal = 2, kPartLJ = 4;

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

__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// The 27 neighbour cells as 9 rows (dz, dy) of three x-adjacent cells.  Cells
// are numbered x fastest, so a row is one contiguous range of the sorted
// particles unless it wraps around the box edge; then it is two ranges.
__device__ __forceinline__ void row_ranges(const int* __restrict__ cs, int base, int cx, int ncd,
                                           int& s0, int& e0, int& s1, int& e1) {
    if (cx > 0 && cx < ncd - 1) {
        s0 = __ldg(cs + base + cx - 1); e0 = __ldg(cs + base + cx + 2); s1 = 0; e1 = 0;
    } else if (cx == 0) {
        s0 = __ldg(cs + base); e0 = __ldg(cs + base + 2);
        s1 = __ldg(cs + base + ncd - 1); e1 = __ldg(cs + base + ncd);
    } else {
        s0 = __ldg(cs + base + ncd - 2); e0 = __ldg(cs + base + ncd);
        s1 = __ldg(cs + base); e1 = __ldg(cs + base + 1);
    }
}

// ----------------------------------------------------------------- mixed
// G threads cooperate on one particle: they stride over the candidates of each
// row, and their partial sums are combined with shuffles.
template <int G>
__global__ void __launch_bounds__(kBlockP)
k_real_mixed(RealArgs a) {
    const Tile tl = a.rblk[blockIdx.x];
    const SysDev& S = a.sys[tl.sys];
    const int g = threadIdx.x % G;
    const int t = threadIdx.x / G;
    const bool active = t < tl.count;
    const int i = tl.first + (tl.count > 0 ? min(t, tl.count - 1) : 0);
    uint4 pi = make_uint4(0, 0, 0, 0);
    if (tl.count > 0) pi = a.spos[i];
    const float qi = __uint_as_float(pi.w);
    const bool do_real = (a.parts & kPartReal) != 0;
    const bool do_lj = (a.parts & kPartLJ) != 0 && S.lj_eps != 0.0;
    float fx = 0.f, fy = 0.f, fz = 0.f, phr = 0.f, ec = 0.f, elj = 0.f;
    if (active && (do_real || do_lj)) {
        const int ncd = S.ncd;
        const int cx = (int)(((unsigned long long)pi.x * ncd) >> 32);
        const int cy = (int)(((unsigned long long)pi.y * ncd) >> 32);
        const int cz = (int)(((unsigned long long)pi.z * ncd) >> 32);
        const float Lu = S.L_over_2_32;
        const float rc2 = do_real ? (float)(S.r_c * S.r_c) : 0.f;
        const float alpha = (float)S.alpha, sa = (float)S.sqrt_alpha;
        const float two_sa_spi = (float)(2.0 * S.sqrt_alpha / sqrt(M_PI));
        const float lB = (float)S.lB;
        const float lj_rc2 = do_lj ? (float)S.lj_rcut2 : 0.f, lj_s2 = (float)S.lj_sigma2;
        const float lj_eps = (float)S.lj_eps, lj_shift = (float)S.lj_shift;
        const float lbqi = lB * qi;
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = wrapc(cz + dz, ncd);
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = wrapc(cy + dy, ncd);
                int s0, e0, s1, e1;
                row_ranges(a.cell_start, S.off_c + (zz * ncd + yy) * ncd, cx, ncd, s0, e0, s1, e1);
#pragma unroll 1
                for (int r = 0; r < 2; ++r) {
                    const int s = r ? s1 : s0, e = r ? e1 : e0;
#pragma unroll 2
                    for (int j = s + g; j < e; j += G) {
                        const uint4 pj = __ldg(a.spos + j);
                        const float ddx = (float)(int32_t)(pj.x - pi.x) * Lu;
                        const float ddy = (float)(int32_t)(pj.y - pi.y) * Lu;
                        const float ddz = (float)(int32_t)(pj.z - pi.z) * Lu;
                        const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                        if (j == i) continue;
                        if (r2 < rc2) {
                            const float qj = __uint_as_float(pj.w);
                            const float inv_r = rsqrtf(r2);
                            const float rr = r2 * inv_r;
                            const float erfc_v = erfcf(sa * rr);
                            const float ex = expf(-alpha * r2);
                            const float pot = erfc_v * inv_r;                 // erfc / r
                            const float g_over_r = fmaf(two_sa_spi, ex, pot) * inv_r * inv_r;
                            const float s_ = -lbqi * qj * g_over_r;
                            fx = fmaf(s_, ddx, fx);
                            fy = fmaf(s_, ddy, fy);
                            fz = fmaf(s_, ddz, fz);
                            phr = fmaf(lB * qj, pot, phr);
                            ec = fmaf(0.5f * lbqi * qj, pot, ec);
                        }
                        if (r2 < lj_rc2) {
                            const float sr2 = lj_s2 / r2;
                            const float sr6 = sr2 * sr2 * sr2;
                            const float mag = 24.f * lj_eps * (2.f * sr6 * sr6 - sr6) / r2;
                            fx = fmaf(-mag, ddx, fx);
                            fy = fmaf(-mag, ddy, fy);
                            fz = fmaf(-mag, ddz, fz);
                            elj += 0.5f * (4.f * lj_eps * (sr6 * sr6 - sr6) + lj_shift);
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o, G);
        fy += __shfl_down_sync(0xffffffffu, fy, o, G);
        fz += __shfl_down_sync(0xffffffffu, fz, o, G);
        phr += __shfl_down_sync(0xffffffffu, phr, o, G);
        ec += __shfl_down_sync(0xffffffffu, ec, o, G);
        elj += __shfl_down_sync(0xffffffffu, elj, o, G);
    }
    const bool owner = active && g == 0;
    if (owner) {
        float phi = phr;
        if (a.parts & kPartFourier) {
            const float4 f = a.fs[i];
            fx += f.x; fy += f.y; fz += f.z;
            const double2 qs = a.qsum[tl.sys];
            phi += f.w - (float)(2.0 * S.self_coef * (double)qi + S.bg_coef * qs.x);
        }
        const int o = a.perm[i];
        if (a.F_out) a.F_out[o] = make_float4(fx, fy, fz, 0.f);
        if (a.phi_out) a.phi_out[o] = phi;
        if (a.md_pos) {
            const uint64_t step = *a.cur_step;
            const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
            const uint4 w = philox4x32_10(
                make_uint4((uint32_t)(o - S.off_p), 0u, (uint32_t)step, (S.stream << 8) | 0x02u),
                key);
            const float u1 = (float)((w.x >> 8) + 1u) * 5.9604644775390625e-08f;   // (0, 1]
            const float u2 = (float)(w.y >> 8) * 5.9604644775390625e-08f;          // [0, 1)
            const float u3 = (float)((w.z >> 8) + 1u) * 5.9604644775390625e-08f;
            const float u4 = (float)(w.w >> 8) * 5.9604644775390625e-08f;
            const float r1 = sqrtf(-2.f * logf(u1)), r3 = sqrtf(-2.f * logf(u3));
            float s2, c2v, s4, c4;
            sincospif(2.f * u2, &s2, &c2v);
            sincospif(2.f * u4, &s4, &c4);
            const float xi0 = r1 * c2v, xi1 = r1 * s2, xi2 = r3 * c4;
            const float c1 = (float)S.c1, c2 = (float)S.c2, dtm = (float)S.dt_over_m;
            const float dt = (float)S.dt;
            float4 v = a.md_vel[o];
            float4 rp = a.md_pos[o];
            v.x = fmaf(c1, fmaf(dtm, fx, v.x), c2 * xi0);
            v.y = fmaf(c1, fmaf(dtm, fy, v.y), c2 * xi1);
            v.z = fmaf(c1, fmaf(dtm, fz, v.z), c2 * xi2);
            const float L = S.Lf, invL = (float)S.invL;
            rp.x = fmaf(dt, v.x, rp.x); rp.x -= L * floorf(rp.x * invL);
            rp.y = fmaf(dt, v.y, rp.y); rp.y -= L * floorf(rp.y * invL);
            rp.z = fmaf(dt, v.z, rp.z); rp.z -= L * floorf(rp.z * invL);
            // a coordinate just below 0 can round up to exactly L: that is 0
            if (rp.x >= L) rp.x = 0.f;
            if (rp.y >= L) rp.y = 0.f;
            if (rp.z >= L) rp.z = 0.f;
            a.md_vel[o] = v;
            a.md_pos[o] = rp;
        }
    }
    if (a.blk_e) {
        const double2 r = block_sum2_real(owner ? (double)ec : 0.0, owner ? (double)elj : 0.0);
        if (threadIdx.x == 0) a.blk_e[blockIdx.x] = r;
    }
}

// ----------------------------------------------------------------- FP64
template <int G>
__global__ void __launch_bounds__(kBlockP)
k_real_f64(RealArgs a) {
    const Tile tl = a.rblk[blockIdx.x];
    const SysDev& S = a.sys[tl.sys];
    const int g = threadIdx.x % G;
    const int t = threadIdx.x / G;
    const bool active = t < tl.count;
    const int i = tl.first + (tl.count > 0 ? min(t, tl.count - 1) : 0);
    double4 pi = make_double4(0, 0, 0, 0);
    if (tl.count > 0) pi = a.spos64[i];
    const double qi = pi.w;
    const bool do_real = (a.parts & kPartReal) != 0;
    const bool do_lj = (a.parts & kPartLJ) != 0 && S.lj_eps != 0.0;
    double fx = 0, fy = 0, fz = 0, phr = 0, ec = 0, elj = 0;
    if (active && (do_real || do_lj)) {
        const int ncd = S.ncd;
        auto cell = [&](double w) {
            const double u = w * S.invL * (double)ncd;
            return (u >= 0.0 && u < (double)ncd) ? (int)u : 0;
        };
        const int cx = cell(pi.x), cy = cell(pi.y), cz = cell(pi.z);
        const double L = S.L, invL = S.invL;
        const double rc2 = do_real ? S.r_c * S.r_c : 0.0;
        const double lj_rc2 = do_lj ? S.lj_rcut2 : 0.0;
        const double two_sa_spi = 2.0 * S.sqrt_alpha / sqrt(M_PI);
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = wrapc(cz + dz, ncd);
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = wrapc(cy + dy, ncd);
                int s0, e0, s1, e1;
                row_ranges(a.cell_start, S.off_c + (zz * ncd + yy) * ncd, cx, ncd, s0, e0, s1, e1);
                for (int r = 0; r < 2; ++r) {
                    const int s = r ? s1 : s0, e = r ? e1 : e0;
                    for (int j = s + g; j < e; j += G) {
                        if (j == i) continue;
                        const double4 pj = a.spos64[j];
                        double ddx = pj.x - pi.x, ddy = pj.y - pi.y, ddz = pj.z - pi.z;
                        ddx -= L * rint(ddx * invL);
                        ddy -= L * rint(ddy * invL);
                        ddz -= L * rint(ddz * invL);
                        const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        if (r2 < rc2) {
                            const double r = sqrt(r2);
                            const double erfc_v = erfc(S.sqrt_alpha * r);
                            const double G_ = erfc_v / r2 + two_sa_spi * exp(-S.alpha * r2) / r;
                            const double s_ = -S.lB * qi * pj.w * G_ / r;
                            fx += s_ * ddx; fy += s_ * ddy; fz += s_ * ddz;
                            phr += S.lB * pj.w * erfc_v / r;
                            ec += 0.5 * S.lB * qi * pj.w * erfc_v / r;
                        }
                        if (r2 < lj_rc2) {
                            const double sr2 = S.lj_sigma2 / r2;
                            const double sr6 = sr2 * sr2 * sr2;
                            const double mag = 24.0 * S.lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                            fx -= mag * ddx; fy -= mag * ddy; fz -= mag * ddz;
                            elj += 0.5 * (4.0 * S.lj_eps * (sr6 * sr6 - sr6) + S.lj_shift);
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o, G);
        fy += __shfl_down_sync(0xffffffffu, fy, o, G);
        fz += __shfl_down_sync(0xffffffffu, fz, o, G);
        phr += __shfl_down_sync(0xffffffffu, phr, o, G);
        ec += __shfl_down_sync(0xffffffffu, ec, o, G);
        elj += __shfl_down_sync(0xffffffffu, elj, o, G);
    }
    const bool owner = active && g == 0;
    if (owner) {
        double phi = phr;
        if (a.parts & kPartFourier) {
            const double4 f = a.fs64[i];
            fx += f.x; fy += f.y; fz += f.z;
            const double2 qs = a.qsum[tl.sys];
            phi += f.w - 2.0 * S.self_coef * qi - S.bg_coef * qs.x;
        }
        const int o = a.perm[i];
        if (a.F_out64) a.F_out64[o] = make_double4(fx, fy, fz, 0.0);
        if (a.phi_out64) a.phi_out64[o] = phi;
        if (a.md_pos64) {
            const uint64_t step = *a.cur_step;
            const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
            const uint4 w = philox4x32_10(
                make_uint4((uint32_t)(o - S.off_p), 0u, (uint32_t)step, (S.stream << 8) | 0x02u),
                key);
            const double u1 = ((double)w.x + 1.0) / 4294967296.0;
            const double u2 = (double)w.y / 4294967296.0;
            const double u3 = ((double)w.z + 1.0) / 4294967296.0;
            const double u4 = (double)w.w / 4294967296.0;
            const double r1 = sqrt(-2.0 * log(u1)), r3 = sqrt(-2.0 * log(u3));
            const double xi[3] = {r1 * cos(2.0 * M_PI * u2), r1 * sin(2.0 * M_PI * u2),
                                  r3 * cos(2.0 * M_PI * u4)};
            const double F3[3] = {fx, fy, fz};
            double4 v = a.md_vel64[o];
            double4 rp = a.md_pos64[o];
            double* vv[3] = {&v.x, &v.y, &v.z};
            double* rr[3] = {&rp.x, &rp.y, &rp.z};
            const double L = S.L;
            for (int d = 0; d < 3; ++d) {
                double vd = *vv[d] + S.dt_over_m * F3[d];
                vd = S.c1 * vd + S.c2 * xi[d];
                double rd = *rr[d] + S.dt * vd;
                rd -= L * floor(rd / L);
                *vv[d] = vd;
                *rr[d] = rd;
            }
            a.md_vel64[o] = v;
            a.md_pos64[o] = rp;
        }
    }
    if (a.blk_e) {
        const double2 r = block_sum2_real(owner ? ec : 0.0, owner ? elj : 0.0);
        if (threadIdx.x == 0) a.blk_e[blockIdx.x] = r;
    }
}

// ----------------------------------------------------------------- energy
// One block per system: fixed-order FP64 sums of the per-k energy terms and the
// per-block real-space / LJ partials, plus the self and background terms.
__global__ void k_energy(const SysDev* __restrict__ sysv, const double* __restrict__ eterm,
                         const double2* __restrict__ blk_e, const double2* __restrict__ qsum,
                         int parts, double* __restrict__ E_out) {
    const SysDev& S = sysv[blockIdx.x];
    double ef = 0.0, ec = 0.0, elj = 0.0;
    if (parts & kPartFourier)
        for (int l = threadIdx.x; l < S.P; l += blockDim.x) ef += eterm[S.off_k + l];
    if (blk_e)
        for (int b = threadIdx.x; b < S.nrb; b += blockDim.x) {
            const double2 v = blk_e[S.off_rb + b];
            ec += v.x;
            elj += v.y;
        }
    __shared__ double sf[256], sc[256], sl[256];
    sf[threadIdx.x] = ef; sc[threadIdx.x] = ec; sl[threadIdx.x] = elj;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sf[threadIdx.x] += sf[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
            sl[threadIdx.x] += sl[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double Ef = 0.0;
        if (parts & kPartFourier) {
            const double2 qs = qsum[blockIdx.x];
            Ef = sf[0] - S.self_coef * qs.y - 0.5 * S.bg_coef * qs.x * qs.x;
        }
        const double Ec = (parts & kPartReal) ? sc[0] : 0.0;
        const double El = (parts & kPartLJ) ? sl[0] : 0.0;
        E_out[4 * blockIdx.x + 0] = Ef + Ec + El;
        E_out[4 * blockIdx.x + 1] = Ef;
        E_out[4 * blockIdx.x + 2] = Ec;
        E_out[4 * blockIdx.x + 3] = El;
    }
}

void launch_real_mixed(cudaStream_t st, const RealArgs& a) {
    if (a.nrblk <= 0) return;
    switch (a.split) {
        case 2: k_real_mixed<2><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 4: k_real_mixed<4><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 8: k_real_mixed<8><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 16: k_real_mixed<16><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 32: k_real_mixed<32><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        default: k_real_mixed<1><<<a.nrblk, kBlockP, 0, st>>>(a); break;
    }
}

void launch_real_f64(cudaStream_t st, const RealArgs& a) {
    if (a.nrblk <= 0) return;
    switch (a.split) {
        case 2: k_real_f64<2><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 4: k_real_f64<4><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 8: k_real_f64<8><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 16: k_real_f64<16><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        case 32: k_real_f64<32><<<a.nrblk, kBlockP, 0, st>>>(a); break;
        default: k_real_f64<1><<<a.nrblk, kBlockP, 0, st>>>(a); break;
    }
}

void launch_energy(cudaStream_t st, const SysDev* sys, int nsys, const double* eterm,
                   const double2* blk_e, const double2* qsum, int parts, double* E_out) {
    if (nsys <= 0) return;
    k_energy<<<nsys, 256, 0, st>>>(sys, eterm, blk_e, qsum, parts, E_out);
}

}  // namespace rbe
