// rbe_fourier.cu -- the Fourier (long-range) part of one RBE evaluation.
//
//  k-sampling   P i.i.d. m in Z^3 \ {0} from P_k ~ exp(-k^2 / 4 alpha)   (Eq. probexpression)
//               by a per-axis integer inverse-CDF table indexed with Philox words;
//  k_rho        per-chunk partial structure factors
//                 rho_chunk(k_l) = sum_{j in chunk} q_j exp(i k_l . r_j)          (Sec. 2)
//               one thread per wave vector, particles staged in shared memory and
//               read as broadcasts; the k-batch is drawn by the same blocks;
//  k_finalize   FP64 sum of the chunk partials in a fixed order -> rho(k_l), the
//               estimator's energy terms (S/P) 2 pi |rho|^2 / (V k^2) and the
//               per-k force coefficients (S/P) 4 pi / (V k^2) * (Im rho, Re rho);
//  k_force      per particle: F*_i = -q_i sum_l coef_l k_l Im(e^{-i k_l.r_i} rho_l)
//               (Eq. rbmapprox) and the Fourier part of dE/dq_i, with the k-batch
//               staged in shared memory.
//
// Mixed path phases: theta = 2 pi (m . s mod 1) with s the 32-bit fixed-point
// fraction of the position; the product is exact in 32-bit integer arithmetic,
// so the only phase error is the conversion of a 32-bit integer to FP32
// (2^-25 turns).  sin/cos then run on the special-function unit for arguments
// in [-pi, pi).  No FP32 work grows with |m| or L.
#include <cmath>

#include "rbe_internal.cuh"

namespace rbe {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;   // 2 pi / 2^32
constexpr int kStage = 512;                                 // particles staged per pass

// Smallest j in [0, n) with w < T[j] (T[n-1] = 2^32 > any w).
__device__ __forceinline__ int axis_lookup(const uint64_t* __restrict__ T, int n, uint32_t w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)w < __ldg(T + mid)) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Sample l of system S at `step`: (m_x, m_y, m_z, attempts).
__device__ __forceinline__ int4 sample_one(const SysDev& S, const uint64_t* __restrict__ T, int l,
                                           uint64_t step, int* err) {
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    const int n = 2 * S.M + 1;
    for (int a = 0; a < kMaxAttempts; ++a) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)l, (uint32_t)a, (uint32_t)step, (S.stream << 8) | 0x01u), key);
        const int mx = axis_lookup(T, n, w.x) - S.M;
        const int my = axis_lookup(T, n, w.y) - S.M;
        const int mz = axis_lookup(T, n, w.z) - S.M;
        if (mx != 0 || my != 0 || mz != 0) return make_int4(mx, my, mz, a + 1);
    }
    atomicOr(err, kErrSampler);
    return make_int4(1, 0, 0, kMaxAttempts + 1);   // keeps later arithmetic finite
}

// As sample_one, with the table's first 2M entries staged in shared memory as
// 32-bit words (entry 2M = 2^32 is implicit).
__device__ __forceinline__ int4 sample_one_smem(const SysDev& S, const uint32_t* __restrict__ T,
                                                int l, uint64_t step, int* err) {
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    const int last = 2 * S.M;
    auto lookup = [&](uint32_t w) {
        int lo = 0, hi = last;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (w < T[mid]) hi = mid; else lo = mid + 1;
        }
        return lo - S.M;
    };
    for (int a = 0; a < kMaxAttempts; ++a) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)l, (uint32_t)a, (uint32_t)step, (S.stream << 8) | 0x01u), key);
        const int mx = lookup(w.x), my = lookup(w.y), mz = lookup(w.z);
        if (mx != 0 || my != 0 || mz != 0) return make_int4(mx, my, mz, a + 1);
    }
    atomicOr(err, kErrSampler);
    return make_int4(1, 0, 0, kMaxAttempts + 1);
}

// Stage the first 2M table entries of system S into shared memory.
__device__ __forceinline__ void stage_table(const SysDev& S, const uint64_t* __restrict__ table,
                                            uint32_t* s_tab) {
    const uint64_t* T = table + S.off_t;
    for (int j = threadIdx.x; j < 2 * S.M; j += blockDim.x) s_tab[j] = (uint32_t)__ldg(T + j);
}

__global__ void k_sample(const SysDev* __restrict__ sysv, int nsys, int ktot,
                         const int* __restrict__ kstart, const uint64_t* __restrict__ table,
                         const uint64_t* __restrict__ cur_step, int4* __restrict__ ksamp,
                         int* __restrict__ err) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ktot) return;
    const int s = find_sys(kstart, nsys, g);
    const SysDev& S = sysv[s];
    ksamp[g] = sample_one(S, table + S.off_t, g - S.off_k, *cur_step, err);
}

// ----------------------------------------------------------------- rho (mixed)
__global__ void __launch_bounds__(kLTile)
k_rho_mixed(const SysDev* __restrict__ sysv, const Tile* __restrict__ chunks, int tab_smem,
            const uint64_t* __restrict__ table, const uint64_t* __restrict__ cur_step,
            const uint4* __restrict__ spos, float2* __restrict__ part, int4* __restrict__ ksamp,
            int* __restrict__ err) {
    __shared__ uint4 sp[kStage];
    extern __shared__ uint32_t s_tab[];
    const Tile ch = chunks[blockIdx.x];
    const SysDev& S = sysv[ch.sys];
    const int l = blockIdx.y * kLTile + threadIdx.x;
    if (blockIdx.y * kLTile >= S.P) return;          // whole block beyond this system's P
    const bool active = l < S.P;
    if (tab_smem) {
        stage_table(S, table, s_tab);
        __syncthreads();
    }
    int4 m = make_int4(0, 0, 0, 0);
    if (active) {
        m = tab_smem ? sample_one_smem(S, s_tab, l, *cur_step, err)
                     : sample_one(S, table + S.off_t, l, *cur_step, err);
        if (ch.aux == S.off_part) ksamp[S.off_k + l] = m;
    }
    const uint32_t mx = (uint32_t)m.x, my = (uint32_t)m.y, mz = (uint32_t)m.z;
    float re = 0.f, im = 0.f;
    for (int base = 0; base < ch.count; base += kStage) {
        const int cnt = min(kStage, ch.count - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) sp[t] = spos[ch.first + base + t];
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const uint4 p = sp[j];
                const uint32_t ph = mx * p.x + my * p.y + mz * p.z;
                const float th = (float)(int32_t)ph * kTwoPiOver2p32;
                float sn, cs;
                __sincosf(th, &sn, &cs);
                const float q = __uint_as_float(p.w);
                re = fmaf(q, cs, re);
                im = fmaf(q, sn, im);
            }
        }
    }
    if (active) part[ch.aux + l] = make_float2(re, im);
}

// ----------------------------------------------------------------- rho (FP64)
__global__ void __launch_bounds__(kLTile)
k_rho_f64(const SysDev* __restrict__ sysv, const Tile* __restrict__ chunks, int tab_smem,
          const uint64_t* __restrict__ table, const uint64_t* __restrict__ cur_step,
          const double4* __restrict__ spos64, double2* __restrict__ part64,
          int4* __restrict__ ksamp, int* __restrict__ err) {
    __shared__ double4 sp[kStage / 2];
    extern __shared__ uint32_t s_tab[];
    const Tile ch = chunks[blockIdx.x];
    const SysDev& S = sysv[ch.sys];
    const int l = blockIdx.y * kLTile + threadIdx.x;
    if (blockIdx.y * kLTile >= S.P) return;
    const bool active = l < S.P;
    if (tab_smem) {
        stage_table(S, table, s_tab);
        __syncthreads();
    }
    int4 m = make_int4(0, 0, 0, 0);
    if (active) {
        m = tab_smem ? sample_one_smem(S, s_tab, l, *cur_step, err)
                     : sample_one(S, table + S.off_t, l, *cur_step, err);
        if (ch.aux == S.off_part) ksamp[S.off_k + l] = m;
    }
    const double tp = 2.0 * M_PI * S.invL;
    const double kx = tp * m.x, ky = tp * m.y, kz = tp * m.z;
    double re = 0.0, im = 0.0;
    for (int base = 0; base < ch.count; base += kStage / 2) {
        const int cnt = min(kStage / 2, ch.count - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) sp[t] = spos64[ch.first + base + t];
        __syncthreads();
        if (active) {
            for (int j = 0; j < cnt; ++j) {
                const double4 p = sp[j];
                const double th = kx * p.x + ky * p.y + kz * p.z;
                double sn, cs;
                sincos(th, &sn, &cs);
                re += p.w * cs;
                im += p.w * sn;
            }
        }
    }
    if (active) part64[ch.aux + l] = make_double2(re, im);
}

// ----------------------------------------------------------------- finalize
// One warp per (system, l): FP64 sum of the system's chunk partials in a fixed
// order; lane 0 writes rho, the energy term and the force coefficients.  The
// last nsys warps sum the per-block (sum q, sum q^2) partials of each system.
__global__ void k_finalize(const SysDev* __restrict__ sysv, int nsys, int ktot,
                           const int* __restrict__ kstart, const float2* __restrict__ part,
                           const double2* __restrict__ part64, const int4* __restrict__ ksamp,
                           double2* __restrict__ rho, float2* __restrict__ kab,
                           double2* __restrict__ kab64, double* __restrict__ eterm,
                           const double2* __restrict__ blk_q, double2* __restrict__ qsum) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < ktot) {
        const int s = find_sys(kstart, nsys, w);
        const SysDev& S = sysv[s];
        const int l = w - S.off_k;
        double re = 0.0, im = 0.0;
        if (part) {
            for (int c = lane; c < S.nchunk; c += 32) {
                const float2 v = part[S.off_part + c * S.P + l];
                re += (double)v.x;
                im += (double)v.y;
            }
        } else {
            for (int c = lane; c < S.nchunk; c += 32) {
                const double2 v = part64[S.off_part + c * S.P + l];
                re += v.x;
                im += v.y;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            const int4 m = ksamp[w];
            const double m2 = (double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z;
            const double tp = 2.0 * M_PI * S.invL;
            const double k2 = tp * tp * m2;
            const double coef = S.coef_scale / k2;        // lB (S/P) 4 pi / (V k^2)
            rho[w] = make_double2(re, im);
            eterm[w] = 0.5 * coef * (re * re + im * im);  // lB (S/P) 2 pi |rho|^2 / (V k^2)
            if (kab) kab[w] = make_float2((float)(coef * im), (float)(coef * re));
            if (kab64) kab64[w] = make_double2(coef * im, coef * re);
        }
    } else if (w < ktot + nsys) {
        const int s = w - ktot;
        const SysDev& S = sysv[s];
        double a = 0.0, b = 0.0;
        if (blk_q) {
            for (int k = lane; k < S.nb; k += 32) {
                const double2 v = blk_q[S.off_b + k];
                a += v.x;
                b += v.y;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) qsum[s] = make_double2(a, b);
    }
}

// ----------------------------------------------------------------- force (mixed)
// Shared-memory record per wave vector: the integer m (phase) and, as floats,
// m (direction) with the two coefficients A = coef Im rho, B = coef Re rho.
struct KPhase { uint32_t mx, my, mz, pad; };
struct KForce { float mx, my, mz, A; };

template <int SPLIT>
__global__ void __launch_bounds__(kBlockP)
k_force_mixed(const SysDev* __restrict__ sysv, const Tile* __restrict__ pblk,
              const uint4* __restrict__ spos, const int4* __restrict__ ksamp,
              const float2* __restrict__ kab, float4* __restrict__ fs) {
    constexpr int kKT = 256;                        // wave vectors staged per pass
    __shared__ KPhase kp[kKT];
    __shared__ KForce kf[kKT];
    __shared__ float kb[kKT];
    constexpr int PER_BLOCK = kBlockP / SPLIT;      // particles per block
    const Tile tl = pblk[blockIdx.x];
    const SysDev& S = sysv[tl.sys];
    const int sub = threadIdx.x % SPLIT;            // lane within the particle's group
    const int t = threadIdx.x / SPLIT;
    const int i = tl.first + min(t, max(tl.count - 1, 0));
    const bool active = t < tl.count;
    uint4 p = make_uint4(0, 0, 0, 0);
    if (tl.count > 0) p = spos[i];
    float fx = 0.f, fy = 0.f, fz = 0.f, ph = 0.f;
    for (int base = 0; base < S.P; base += kKT) {
        const int cnt = min(kKT, S.P - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int4 m = ksamp[S.off_k + base + k];
            const float2 ab = kab[S.off_k + base + k];
            kp[k] = KPhase{(uint32_t)m.x, (uint32_t)m.y, (uint32_t)m.z, 0u};
            kf[k] = KForce{(float)m.x, (float)m.y, (float)m.z, ab.x};
            kb[k] = ab.y;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = sub; k < cnt; k += SPLIT) {
            const KPhase a = kp[k];
            const uint32_t phs = a.mx * p.x + a.my * p.y + a.mz * p.z;
            const float th = (float)(int32_t)phs * kTwoPiOver2p32;
            float sn, cs;
            __sincosf(th, &sn, &cs);
            const KForce f = kf[k];
            const float B = kb[k];
            const float g = fmaf(cs, f.A, -sn * B);     // Im(e^{-i th} rho) * coef
            fx = fmaf(g, f.mx, fx);
            fy = fmaf(g, f.my, fy);
            fz = fmaf(g, f.mz, fz);
            ph = fmaf(cs, B, fmaf(sn, f.A, ph));        // Re(e^{-i th} rho) * coef
        }
    }
#pragma unroll
    for (int o = SPLIT / 2; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o, SPLIT);
        fy += __shfl_down_sync(0xffffffffu, fy, o, SPLIT);
        fz += __shfl_down_sync(0xffffffffu, fz, o, SPLIT);
        ph += __shfl_down_sync(0xffffffffu, ph, o, SPLIT);
    }
    (void)PER_BLOCK;
    if (active && sub == 0) {
        const float q = __uint_as_float(p.w);
        const float sc = -q * (float)(2.0 * M_PI) * (float)S.invL;
        fs[i] = make_float4(sc * fx, sc * fy, sc * fz, ph);
    }
}

// ----------------------------------------------------------------- force (FP64)
__global__ void __launch_bounds__(kBlockP)
k_force_f64(const SysDev* __restrict__ sysv, const Tile* __restrict__ pblk,
            const double4* __restrict__ spos64, const int4* __restrict__ ksamp,
            const double2* __restrict__ kab64, double4* __restrict__ fs64) {
    constexpr int kKT = 256;
    __shared__ double4 kk[kKT];     // kx, ky, kz, A
    __shared__ double kb[kKT];      // B
    const Tile tl = pblk[blockIdx.x];
    const SysDev& S = sysv[tl.sys];
    const int t = threadIdx.x;
    const bool active = t < tl.count;
    double4 p = make_double4(0, 0, 0, 0);
    if (active) p = spos64[tl.first + t];
    const double tp = 2.0 * M_PI * S.invL;
    double fx = 0, fy = 0, fz = 0, ph = 0;
    for (int base = 0; base < S.P; base += kKT) {
        const int cnt = min(kKT, S.P - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int4 m = ksamp[S.off_k + base + k];
            const double2 ab = kab64[S.off_k + base + k];
            kk[k] = make_double4(tp * m.x, tp * m.y, tp * m.z, ab.x);
            kb[k] = ab.y;
        }
        __syncthreads();
        if (active) {
            for (int k = 0; k < cnt; ++k) {
                const double4 kv = kk[k];
                const double th = kv.x * p.x + kv.y * p.y + kv.z * p.z;
                double sn, cs;
                sincos(th, &sn, &cs);
                const double B = kb[k];
                const double g = cs * kv.w - sn * B;
                fx += g * kv.x;
                fy += g * kv.y;
                fz += g * kv.z;
                ph += cs * B + sn * kv.w;
            }
        }
    }
    if (active) fs64[tl.first + t] = make_double4(-p.w * fx, -p.w * fy, -p.w * fz, ph);
}

// ------------------------------------------------------------- launchers
void launch_sample(cudaStream_t st, const SysDev* sys, int nsys, int ktot, const int* kstart,
                   const uint64_t* table, const uint64_t* cur_step, int4* ksamp, int* err) {
    if (ktot <= 0) return;
    k_sample<<<(ktot + 127) / 128, 128, 0, st>>>(sys, nsys, ktot, kstart, table, cur_step, ksamp,
                                                 err);
}

// tab_smem: number of 32-bit table entries to stage per block (max 2M over the
// systems), 0 to search the table in global memory.
void launch_rho_mixed(cudaStream_t st, const SysDev* sys, const Tile* chunks, int nchunks,
                      int ltiles, int tab_smem, const uint64_t* table, const uint64_t* cur_step,
                      const uint4* spos, float2* part, int4* ksamp, int* err) {
    if (nchunks <= 0 || ltiles <= 0) return;
    dim3 grid(nchunks, ltiles);
    k_rho_mixed<<<grid, kLTile, sizeof(uint32_t) * tab_smem, st>>>(
        sys, chunks, tab_smem > 0 ? 1 : 0, table, cur_step, spos, part, ksamp, err);
}

void launch_rho_f64(cudaStream_t st, const SysDev* sys, const Tile* chunks, int nchunks,
                    int ltiles, int tab_smem, const uint64_t* table, const uint64_t* cur_step,
                    const double4* spos64, double2* part64, int4* ksamp, int* err) {
    if (nchunks <= 0 || ltiles <= 0) return;
    dim3 grid(nchunks, ltiles);
    k_rho_f64<<<grid, kLTile, sizeof(uint32_t) * tab_smem, st>>>(
        sys, chunks, tab_smem > 0 ? 1 : 0, table, cur_step, spos64, part64, ksamp, err);
}

void launch_finalize(cudaStream_t st, const SysDev* sys, int nsys, int ktot, const int* kstart,
                     const float2* part, const double2* part64, const int4* ksamp,
                     double2* rho, float2* kab, double2* kab64, double* eterm,
                     const double2* blk_q, double2* qsum) {
    const int warps = ktot + nsys;
    if (warps <= 0) return;
    const int threads = 64;          // few warps per block: spread the FP64 sums over all SMs
    const int blocks = (warps * 32 + threads - 1) / threads;
    k_finalize<<<blocks, threads, 0, st>>>(sys, nsys, ktot, kstart, part, part64, ksamp, rho,
                                           kab, kab64, eterm, blk_q, qsum);
}

void launch_fourier_force_mixed(cudaStream_t st, const SysDev* sys, const Tile* pblk, int npblk,
                                int split, const uint4* spos, const int4* ksamp,
                                const float2* kab, float4* fs) {
    if (npblk <= 0) return;
    switch (split) {
        case 2: k_force_mixed<2><<<npblk, kBlockP, 0, st>>>(sys, pblk, spos, ksamp, kab, fs); break;
        case 4: k_force_mixed<4><<<npblk, kBlockP, 0, st>>>(sys, pblk, spos, ksamp, kab, fs); break;
        case 8: k_force_mixed<8><<<npblk, kBlockP, 0, st>>>(sys, pblk, spos, ksamp, kab, fs); break;
        default: k_force_mixed<1><<<npblk, kBlockP, 0, st>>>(sys, pblk, spos, ksamp, kab, fs); break;
    }
}

void launch_fourier_force_f64(cudaStream_t st, const SysDev* sys, const Tile* pblk, int npblk,
                              const double4* spos64, const int4* ksamp, const double2* kab64,
                              double4* fs64) {
    if (npblk <= 0) return;
    k_force_f64<<<npblk, kBlockP, 0, st>>>(sys, pblk, spos64, ksamp, kab64, fs64);
}

}  // namespace rbe
