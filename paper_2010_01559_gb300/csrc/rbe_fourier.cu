// rbe_fourier.cu -- the Fourier (long-range) part of one RBE evaluation.
//
//  k-sampling   P i.i.d. m in Z^3 \ {0} from P_k ~ exp(-k^2 / 4 alpha)   (Eq. probexpression)
//               by a per-axis integer inverse-CDF table indexed with Philox words;
//  k_rho        per-chunk partial structure factors
//                 rho_chunk(k_l) = sum_{j in chunk} q_j exp(i k_l . r_j)          (Sec. 2)
//               one thread per wave vector, particles (caller's order, so this
//               branch does not wait for the cell sort) staged in shared memory
//               and read as broadcasts; the k-batch is drawn by the same blocks;
//               Each block adds its chunk's partial to rho(k_l) with 64-bit
//               fixed-point atomics: integer addition is associative, so the
//               cross-block sum is bitwise reproducible, with no separate
//               reduction pass;
//  k_force      per particle: F*_i = -q_i sum_l coef_l k_l Im(e^{-i k_l.r_i} rho_l)
//               (Eq. rbmapprox) and the Fourier part of dE/dq_i, with the k-batch
//               and coef_l rho_l, coef_l = (S/P) 4 pi / (V k^2) formed in FP64, staged
//               in shared memory; the mixed path holds coef_l rho_l in polar form
//               (R_l, phi_l), so that an MD step's force takes one sine per pair.
//
// Mixed path phases: theta = 2 pi (m . s mod 1) with s the 32-bit fixed-point
// fraction of the position; the product is exact in 32-bit integer arithmetic,
// so the only phase error is the conversion of a 32-bit integer to FP32
// (2^-25 turns).  sin/cos then run on the special-function unit for arguments
// in [-pi, pi).  No FP32 work grows with |m| or L.
#include <algorithm>
#include <cmath>

#include "rbe_internal.cuh"
#include "rbe_list_body.cuh"

namespace rbe {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;   // 2 pi / 2^32
constexpr int kStage = 512;                                 // particles staged per pass

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

// Force coefficients of wave vector m: coef = lB (S/P) 4 pi / (V k^2) times
// (Im rho, Re rho), from the fixed-point rho(k) accumulator, in FP64.
__device__ __forceinline__ double2 kcoef(const SysDev& S, int4 m,
                                         const unsigned long long* __restrict__ rho) {
    const double2 r = rho_read(rho, S.rho_inv_scale);
    const double tp = 2.0 * M_PI * S.invL;
    const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
    const double coef = S.coef_scale / k2;
    return make_double2(coef * r.y, coef * r.x);
}

// ----------------------------------------------------------------- rho (mixed)
// Two threads per wave vector (threads t and t + kLTile), each over every
// other particle of the chunk; their sums are added before the atomics.
constexpr int kRhoHalves = 2;

// rho_body: chunk ctile of the particles and tile ktile of kRhoKT wave
// vectors (HALVES * kLTile threads; it synchronises the block), for the kernel
// of its own and for the fused structure-factor + list launch of the MD step.
// Each thread takes kRhoK wave vectors, t and t + kLTile of the tile, so that
// one shared-memory load of a particle serves kRhoK (particle, k) pairs.
// With one thread per wave vector (HALVES = 1) the even and odd particles go
// to separate sums that are added as the two halves' are: rho(k) comes out the
// same to the last bit either way.
template <bool ONE, int HALVES>
__device__ __forceinline__ void rho_body(const Work& w, const int4* __restrict__ ksamp,
                                         const double* __restrict__ kcoef,
                                         const uint4* __restrict__ fx,
                                         unsigned long long* __restrict__ rho_fx,
                                         int* __restrict__ kcnt, float2* __restrict__ kab,
                                         int ctile, int ktile) {
    constexpr int KR = kRhoK;
    __shared__ uint4 sp[kStage];
    __shared__ double2 s_half[HALVES > 1 ? kLTile * KR : 1];
    const Tile ch = tile_at<ONE>(w, ctile);
    const SysDev& S = sys_of<ONE>(w, ch.sys);
    const int half = threadIdx.x / kLTile;
    const int t = threadIdx.x - half * kLTile;
    if (ktile * kRhoKT >= S.P) return;               // whole block beyond this system's P
    uint32_t mx[KR], my[KR], mz[KR];
    bool active[KR];
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        const int l = ktile * kRhoKT + t + r * kLTile;
        active[r] = l < S.P;
        int4 m = make_int4(0, 0, 0, 0);
        if (active[r]) m = ksamp[S.off_k + l];       // drawn by the prep kernel
        mx[r] = (uint32_t)m.x;
        my[r] = (uint32_t)m.y;
        mz[r] = (uint32_t)m.z;
    }
    // FP32 sums over one staged pass (at most kStage / 2 terms), FP64 across
    // passes and halves, so the rounding does not grow with the chunk size
    double red[KR], imd[KR], red_o[KR], imd_o[KR];
#pragma unroll
    for (int r = 0; r < KR; ++r) red[r] = imd[r] = red_o[r] = imd_o[r] = 0.0;
    float re[KR], im[KR], re_o[KR], im_o[KR];
    auto terms = [&](const uint4 p, float* re_, float* im_) {
        const float q = __uint_as_float(p.w);
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            const uint32_t ph = mx[r] * p.x + my[r] * p.y + mz[r] * p.z;
            const float th = (float)(int32_t)ph * kTwoPiOver2p32;
            float sn, cs;
            __sincosf(th, &sn, &cs);
            re_[r] = fmaf(q, cs, re_[r]);
            im_[r] = fmaf(q, sn, im_[r]);
        }
    };
    const bool any = active[0];                      // t + kLTile < P only if t < P
    for (int base = 0; base < ch.count; base += kStage) {
        const int cnt = min(kStage, ch.count - base);
        __syncthreads();
        for (int u = threadIdx.x; u < cnt; u += blockDim.x) sp[u] = fx[ch.first + base + u];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < KR; ++r) re[r] = im[r] = re_o[r] = im_o[r] = 0.f;
        if (any) {
            if constexpr (HALVES == 1) {
                int j = 0;
#pragma unroll 8
                for (; j + 1 < cnt; j += 2) {
                    terms(sp[j], re, im);
                    terms(sp[j + 1], re_o, im_o);
                }
                if (j < cnt) terms(sp[j], re, im);
            } else {
#pragma unroll 2
                for (int j = half; j < cnt; j += HALVES) terms(sp[j], re, im);
            }
        }
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            red[r] += (double)re[r];
            imd[r] += (double)im[r];
            red_o[r] += (double)re_o[r];
            imd_o[r] += (double)im_o[r];
        }
    }
    if constexpr (HALVES > 1) {
        if (half == 1) {
#pragma unroll
            for (int r = 0; r < KR; ++r) s_half[t + r * kLTile] = make_double2(red[r], imd[r]);
        }
        __syncthreads();
        if (half == 0) {
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const double2 o = s_half[t + r * kLTile];
                if (active[r])
                    rho_accumulate(rho_fx + 2 * (S.off_k + ktile * kRhoKT + t + r * kLTile),
                                   red[r] + o.x, imd[r] + o.y, S.rho_scale);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < KR; ++r)
            if (active[r])
                rho_accumulate(rho_fx + 2 * (S.off_k + ktile * kRhoKT + t + r * kLTile),
                               red[r] + red_o[r], imd[r] + imd_o[r], S.rho_scale);
    }
    // The last of the system's chunks to add its partials for this tile of
    // wave vectors finds rho(k) complete and turns it into the force
    // coefficient of Eq. rbmapprox in polar form, once per k instead of once
    // per force block: with A = coef Im rho and B = coef Re rho,
    // A cos(theta) - B sin(theta) = R sin(phi - theta) for R = |(A, B)| and
    // phi = atan2(A, B), stored as (R, phi in 2^-32 turns).  Fence, then
    // count: every chunk's atomics are visible to the block that takes the
    // last count (no waiting on other blocks).
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    const int slot = S.off_k + ktile * kRhoKT;
    if (threadIdx.x == 0) s_last = atomicAdd(kcnt + slot, 1) == S.nchunk - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int u = threadIdx.x; u < kRhoKT; u += blockDim.x) {
            const int l = ktile * kRhoKT + u;
            if (l >= S.P) break;
            const double2 r = rho_read(rho_fx + 2 * (S.off_k + l), S.rho_inv_scale);
            const double c = kcoef[S.off_k + l];
            const float A = (float)(c * r.y), B = (float)(c * r.x);
            const float turns = atan2f(A, B) * 0.15915494309189535f;      // (-1/2, 1/2]
            const uint32_t phi = (uint32_t)(long long)llrintf(turns * 4294967296.0f);
            kab[S.off_k + l] = make_float2(hypotf(A, B), __uint_as_float(phi));
        }
        if (threadIdx.x == 0) kcnt[slot] = 0;        // ready for the next evaluation
    }
}

template <bool ONE>
__global__ void __launch_bounds__(kLTile * kRhoHalves)
k_rho_mixed(const __grid_constant__ Work w, const int4* __restrict__ ksamp,
            const double* __restrict__ kcoef, const uint4* __restrict__ fx,
            unsigned long long* __restrict__ rho_fx, int* __restrict__ kcnt,
            float2* __restrict__ kab) {
    pdl_trigger();                                    // the force kernel may be scheduled
    pdl_wait();                                       // the prep kernel's samples and records
    rho_body<ONE, kRhoHalves>(w, ksamp, kcoef, fx, rho_fx, kcnt, kab, blockIdx.x, blockIdx.y);
}

// ------------------------------------------- structure factors + list pass
// The MD step's structure factors and its real-space pass over a standing
// neighbour list in one launch of kLTile-thread blocks: block b takes
// structure-factor work when floor((b + 1) nrho / total) > floor(b nrho /
// total), else a tile of the list pass, so that the two kinds are spread evenly
// over the grid and each SM holds both at once -- the structure factors keep
// the special-function unit busy while the pair terms use the ALU and FMA
// pipes and wait on their gathers.  The list tiles work only when the list
// stands (over a rebuilt list the pass runs on the rebuild stream, after the
// build), and keep the per-slot count tests: padded batches cost this
// issue-bound launch more than they save.
template <int R, bool ONE>
__global__ void __launch_bounds__(kLTile)
k_rho_list(const __grid_constant__ Work w, const int4* __restrict__ ksamp,
           const double* __restrict__ kcoef, const uint4* __restrict__ fx,
           unsigned long long* __restrict__ rho_fx, int* __restrict__ kcnt,
           float2* __restrict__ kab, const __grid_constant__ RealArgs a, int nchunks, int nrho,
           int nlist) {
    pdl_trigger();                                    // the force kernel may be scheduled
    pdl_wait();                                       // the prep kernel's samples and records
    const int b = blockIdx.x, total = nrho + nlist;
    const int r0 = (int)((long long)b * nrho / total);
    const int r1 = (int)((long long)(b + 1) * nrho / total);
    if (r1 > r0) {
        rho_body<ONE, 1>(w, ksamp, kcoef, fx, rho_fx, kcnt, kab, r0 % nchunks, r0 / nchunks);
        return;
    }
    if ((*a.list_flag != 0) != (a.list_when != 0)) return;
    list_body<R, ONE, false, false, 8>(a, b - r1, threadIdx.x);
}

// ----------------------------------------------------------------- rho (FP64)
template <bool ONE>
__global__ void __launch_bounds__(kLTile)
k_rho_f64(const __grid_constant__ Work w, const int4* __restrict__ ksamp,
          const double4* __restrict__ fx64, unsigned long long* __restrict__ rho_fx) {
    __shared__ double4 sp[kStage / 2];
    const Tile ch = tile_of<ONE>(w);
    const SysDev& S = sys_of<ONE>(w, ch.sys);
    const int l = blockIdx.y * kLTile + threadIdx.x;
    if (blockIdx.y * kLTile >= S.P) return;
    const bool active = l < S.P;
    int4 m = make_int4(0, 0, 0, 0);
    if (active) m = ksamp[S.off_k + l];
    const double tp = 2.0 * M_PI * S.invL;
    const double kx = tp * m.x, ky = tp * m.y, kz = tp * m.z;
    double re = 0.0, im = 0.0;
    for (int base = 0; base < ch.count; base += kStage / 2) {
        const int cnt = min(kStage / 2, ch.count - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) sp[t] = fx64[ch.first + base + t];
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
    if (active) rho_accumulate(rho_fx + 2 * (S.off_k + l), re, im, S.rho_scale);
}

// ----------------------------------------------------------------- force (mixed)
// Shared-memory record per wave vector: -m and phi (the phase of the
// coefficient, 2^-32 turns) as integers, and R m (the direction scaled by the
// coefficient's magnitude) with R as floats.  phi - m.s is exact in 32-bit
// arithmetic, so one sine per (particle, k) pair gives the force term
// R m sin(phi - theta) = m coef Im(e^{-i k.r} rho) (and the cosine, in the
// same SFU pair, the dE/dq term R cos(phi - theta)).
struct KPhase { uint32_t nmx, nmy, nmz, phi; };
struct KForce { float rmx, rmy, rmz, R; };

// SPLIT threads per particle (each a 1/SPLIT share of the wave vectors), or
// with SPLIT = 1 PT = 2 particles per thread, which share each wave vector's
// shared-memory loads and the loop overhead (the pass is issue-bound at large
// N).  A block holds a tile of kBlockP / SPLIT particles and kBlockP / PT
// threads.  PHI: also dE/dq (the forces path); MD steps need only the force.
template <int SPLIT, int PT, bool PHI, bool ONE>
__global__ void __launch_bounds__(kBlockP / PT)
k_force_mixed(const __grid_constant__ Work w, const uint4* __restrict__ rec,
              const int4* __restrict__ ksamp, const float2* __restrict__ kab,
              float4* __restrict__ fs, const __grid_constant__ MdOut md) {
    static_assert(PT == 1 || SPLIT == 1, "two particles per thread only with one thread each");
    constexpr int NT = kBlockP / PT;                // threads per block
    constexpr int TILE = kBlockP / SPLIT;           // particles per block
    constexpr int EP = (TILE + NT - 1) / NT;        // closing updates per thread
    constexpr int kKT = 256;                        // wave vectors staged per pass
    __shared__ KPhase kp[kKT];
    __shared__ KForce kf[kKT];
    const Tile tl = tile_of<ONE>(w);
    const SysDev& S = sys_of<ONE>(w, tl.sys);
    const int sub = threadIdx.x % SPLIT;            // lane within the particle's group
    pdl_wait();                                     // rho(k), kab and the real-space forces
    int tq[PT];
    uint4 p[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        tq[q] = threadIdx.x / SPLIT + q * (NT / SPLIT);
        p[q] = make_uint4(0, 0, 0, 0);
        if (tl.count > 0) p[q] = rec[tl.first + min(tq[q], tl.count - 1)];
    }
    // neighbour-list MD step: the inputs of the closing update (thread t:
    // particles t, t + NT, .. of the tile) and the thermostat's noise, fetched
    // before the wave-vector loop -- nothing writes them during this kernel
    const bool nhm = md.md_pos && md.nh && S.thermostat == RBE_THERMO_NOSE_HOOVER;
    float4 e_fr[EP], e_v[EP], e_r[EP];
    MdNoise e_z[EP];
#pragma unroll
    for (int e = 0; e < EP; ++e) {
        e_fr[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        e_v[e] = e_fr[e];
        e_r[e] = e_fr[e];
        e_z[e] = MdNoise{0.f, 0.f, 0.f, false};
        const int te = threadIdx.x + e * NT;
        if (md.freal && te < tl.count) {
            const int o = tl.first + te;
            e_fr[e] = md.freal[o];
            if (md.md_pos) {
                e_v[e] = md.md_vel[o];
                e_r[e] = md.md_pos[o];
                if (!nhm) e_z[e] = md_noise(S, *md.cur_step, o);
            }
        }
    }
    float fx[PT], fy[PT], fz[PT], ph[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) fx[q] = fy[q] = fz[q] = ph[q] = 0.f;
    for (int base = 0; base < S.P; base += kKT) {
        const int cnt = min(kKT, S.P - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int4 m = ksamp[S.off_k + base + k];
            const float2 rp = kab[S.off_k + base + k];
            kp[k] = KPhase{0u - (uint32_t)m.x, 0u - (uint32_t)m.y, 0u - (uint32_t)m.z,
                           __float_as_uint(rp.y)};
            kf[k] = KForce{rp.x * (float)m.x, rp.x * (float)m.y, rp.x * (float)m.z, rp.x};
        }
        __syncthreads();
#pragma unroll 8
        for (int k = sub; k < cnt; k += SPLIT) {
            const KPhase a = kp[k];
            const KForce f = kf[k];
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const uint32_t d = a.phi + a.nmx * p[q].x + a.nmy * p[q].y + a.nmz * p[q].z;
                const float t = (float)(int32_t)d * kTwoPiOver2p32;          // phi - theta
                float sn;                                   // Im(e^{-i theta} rho) coef / R
                if constexpr (PHI) {
                    float cs;
                    __sincosf(t, &sn, &cs);
                    ph[q] = fmaf(f.R, cs, ph[q]);           // Re(e^{-i theta} rho) * coef
                } else {
                    sn = __sinf(t);
                }
                fx[q] = fmaf(sn, f.rmx, fx[q]);
                fy[q] = fmaf(sn, f.rmy, fy[q]);
                fz[q] = fmaf(sn, f.rmz, fz[q]);
            }
        }
    }
#pragma unroll
    for (int o = SPLIT / 2; o > 0; o >>= 1) {
        fx[0] += __shfl_down_sync(0xffffffffu, fx[0], o, SPLIT);
        fy[0] += __shfl_down_sync(0xffffffffu, fy[0], o, SPLIT);
        fz[0] += __shfl_down_sync(0xffffffffu, fz[0], o, SPLIT);
        ph[0] += __shfl_down_sync(0xffffffffu, ph[0], o, SPLIT);
    }
    if (!md.freal) {
#pragma unroll
        for (int q = 0; q < PT; ++q)
            if (tq[q] < tl.count && sub == 0) {
                const float qc = __uint_as_float(p[q].w);
                const float sc = -qc * (float)(2.0 * M_PI) * S.f_invL;
                fs[tl.first + tq[q]] = make_float4(sc * fx[q], sc * fy[q], sc * fz[q], ph[q]);
            }
        return;
    }
    // neighbour-list MD step: the total force and the thermostat
    if (md.list_flag && blockIdx.x == 0 && threadIdx.x == 0) *md.list_flag = 0;   // consumed
    __shared__ float4 s_t[TILE];
#pragma unroll
    for (int q = 0; q < PT; ++q)
        if (tq[q] < tl.count && sub == 0) {
            const float qc = __uint_as_float(p[q].w);
            const float sc = -qc * (float)(2.0 * M_PI) * S.f_invL;
            s_t[tq[q]] = make_float4(sc * fx[q], sc * fy[q], sc * fz[q], 0.f);
        }
    __syncthreads();
    unsigned long long k2 = 0ull;
#pragma unroll
    for (int e = 0; e < EP; ++e) {
        const int te = threadIdx.x + e * NT;
        if (te < tl.count) {
            const int o = tl.first + te;
            const float4 ff = s_t[te];
            const float Fx = e_fr[e].x + ff.x, Fy = e_fr[e].y + ff.y, Fz = e_fr[e].z + ff.z;
            if (md.F_out) md.F_out[o] = make_float4(Fx, Fy, Fz, 0.f);
            if (md.md_pos) {
                if (nhm)
                    k2 += nose_hoover_apply(S, md.nh[tl.sys].f_va, md.nh[tl.sys].f_vf, Fx, Fy,
                                            Fz, e_v[e], e_r[e]);
                else
                    md_apply(S, e_z[e], Fx, Fy, Fz, e_v[e], e_r[e]);
                md.md_vel[o] = e_v[e];
                md.md_pos[o] = e_r[e];
            }
        }
    }
    if (nhm) warp_add_u64(k2, &md.nh[tl.sys].k2);
    if (md.done_host) {
        __threadfence_system();                     // this thread's pos / vel stores
        __syncthreads();
        if (threadIdx.x == 0 && atomicAdd(md.done_cnt, 1u) == gridDim.x - 1) {
            __threadfence_system();                 // every block's stores, then the words
            *md.done_cnt = 0u;
            *(volatile int*)md.err_host = *(const volatile int*)md.err;
            __threadfence_system();
            *(volatile unsigned long long*)md.done_host = *md.cur_step + 1ull;
        }
    }
}

// ----------------------------------------------------------------- force (FP64)
template <bool ONE>
__global__ void __launch_bounds__(kBlockP)
k_force_f64(const __grid_constant__ Work w, const double4* __restrict__ rec64,
            const int4* __restrict__ ksamp, const unsigned long long* __restrict__ rho_fx,
            double4* __restrict__ fs64) {
    constexpr int kKT = 256;
    __shared__ double4 kk[kKT];     // kx, ky, kz, A
    __shared__ double kb[kKT];      // B
    const Tile tl = tile_of<ONE>(w);
    const SysDev& S = sys_of<ONE>(w, tl.sys);
    const int t = threadIdx.x;
    const bool active = t < tl.count;
    double4 p = make_double4(0, 0, 0, 0);
    if (active) p = rec64[tl.first + t];
    const double tp = 2.0 * M_PI * S.invL;
    double fx = 0, fy = 0, fz = 0, ph = 0;
    for (int base = 0; base < S.P; base += kKT) {
        const int cnt = min(kKT, S.P - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int4 m = ksamp[S.off_k + base + k];
            const double2 ab = kcoef(S, m, rho_fx + 2 * (S.off_k + base + k));
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

// The k-batch (ksamp) and coef_scale / k^2 (kcoef) come from the prep kernel.
// A launch configuration, with programmatic stream serialisation if pdl.
struct PdlConfig {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1]{};
    PdlConfig(dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl) {
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pdl ? 1 : 0;
    }
};

void launch_rho_mixed(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                      const int4* ksamp, const double* kcoef, const uint4* fx,
                      unsigned long long* rho_fx, int* kcnt, float2* kab, bool pdl) {
    if (nchunks <= 0 || ltiles <= 0) return;
    PdlConfig c(dim3(nchunks, ltiles), dim3(kLTile * kRhoHalves), 0, st, pdl);
    if (one)
        cudaLaunchKernelEx(&c.cfg, k_rho_mixed<true>, w, ksamp, kcoef, fx, rho_fx, kcnt, kab);
    else
        cudaLaunchKernelEx(&c.cfg, k_rho_mixed<false>, w, ksamp, kcoef, fx, rho_fx, kcnt, kab);
}

template <int R>
static void rho_list_r(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                       const int4* ksamp, const double* kcoef, const uint4* fx,
                       unsigned long long* rho_fx, int* kcnt, float2* kab, const RealArgs& a,
                       bool pdl) {
    const int nrho = nchunks * ltiles;
    PdlConfig c(dim3(nrho + a.nlblk), dim3(kLTile), 0, st, pdl);
    if (one)
        cudaLaunchKernelEx(&c.cfg, k_rho_list<R, true>, w, ksamp, kcoef, fx, rho_fx, kcnt, kab, a,
                           nchunks, nrho, a.nlblk);
    else
        cudaLaunchKernelEx(&c.cfg, k_rho_list<R, false>, w, ksamp, kcoef, fx, rho_fx, kcnt, kab,
                           a, nchunks, nrho, a.nlblk);
}

void launch_rho_list(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                     const int4* ksamp, const double* kcoef, const uint4* fx,
                     unsigned long long* rho_fx, int* kcnt, float2* kab, const RealArgs& a,
                     bool pdl) {
    if (nchunks <= 0 || ltiles <= 0) return;
    switch (a.lsplit) {
        case 2: rho_list_r<2>(st, one, w, nchunks, ltiles, ksamp, kcoef, fx, rho_fx, kcnt, kab, a, pdl); break;
        case 4: rho_list_r<4>(st, one, w, nchunks, ltiles, ksamp, kcoef, fx, rho_fx, kcnt, kab, a, pdl); break;
        case 8: rho_list_r<8>(st, one, w, nchunks, ltiles, ksamp, kcoef, fx, rho_fx, kcnt, kab, a, pdl); break;
        default: rho_list_r<1>(st, one, w, nchunks, ltiles, ksamp, kcoef, fx, rho_fx, kcnt, kab, a, pdl); break;
    }
}

void launch_rho_f64(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                    const int4* ksamp, const double4* fx64, unsigned long long* rho_fx) {
    if (nchunks <= 0 || ltiles <= 0) return;
    dim3 grid(nchunks, ltiles);
    if (one)
        k_rho_f64<true><<<grid, kLTile, 0, st>>>(w, ksamp, fx64, rho_fx);
    else
        k_rho_f64<false><<<grid, kLTile, 0, st>>>(w, ksamp, fx64, rho_fx);
}

template <int SPLIT, int PT>
static void force_mixed_split(cudaStream_t st, bool one, const Work& w, int nblk, const uint4* fx,
                              const int4* ksamp, const float2* kab, float4* fs,
                              const MdOut& md, bool pdl) {
    PdlConfig c(dim3(nblk), dim3(kBlockP / PT), 0, st, pdl);
    if (md.freal) {
        if (one) cudaLaunchKernelEx(&c.cfg, k_force_mixed<SPLIT, PT, false, true>, w, fx, ksamp, kab, fs, md);
        else cudaLaunchKernelEx(&c.cfg, k_force_mixed<SPLIT, PT, false, false>, w, fx, ksamp, kab, fs, md);
    } else {
        if (one) cudaLaunchKernelEx(&c.cfg, k_force_mixed<SPLIT, PT, true, true>, w, fx, ksamp, kab, fs, md);
        else cudaLaunchKernelEx(&c.cfg, k_force_mixed<SPLIT, PT, true, false>, w, fx, ksamp, kab, fs, md);
    }
}

void launch_fourier_force_mixed(cudaStream_t st, bool one, const Work& w, int nblk, int split,
                                const uint4* fx, const int4* ksamp, const float2* kab,
                                float4* fs, const MdOut& md, bool pdl) {
    if (nblk <= 0) return;
    switch (split) {
        case 2: force_mixed_split<2, 1>(st, one, w, nblk, fx, ksamp, kab, fs, md, pdl); break;
        case 4: force_mixed_split<4, 1>(st, one, w, nblk, fx, ksamp, kab, fs, md, pdl); break;
        case 8: force_mixed_split<8, 1>(st, one, w, nblk, fx, ksamp, kab, fs, md, pdl); break;
        default: force_mixed_split<1, 2>(st, one, w, nblk, fx, ksamp, kab, fs, md, pdl); break;
    }
}

void launch_fourier_force_f64(cudaStream_t st, bool one, const Work& w, int nblk,
                              const double4* fx64, const int4* ksamp,
                              const unsigned long long* rho_fx, double4* fs64) {
    if (nblk <= 0) return;
    if (one)
        k_force_f64<true><<<nblk, kBlockP, 0, st>>>(w, fx64, ksamp, rho_fx, fs64);
    else
        k_force_f64<false><<<nblk, kBlockP, 0, st>>>(w, fx64, ksamp, rho_fx, fs64);
}

}  // namespace rbe

namespace rbe {

// ----------------------------------------------------------------- observables
// Full (non-random) Ewald structure factors of one system over a half space of
// wave vectors (m and -m give conjugate rho(k)): the phases as in the
// structure-factor pass (exact 32-bit phase, FP32 sin/cos), the sums in the
// 64-bit fixed-point accumulators.  Grid: (particle chunks, k tiles).
__global__ void __launch_bounds__(kLTile)
k_struct_full(const uint4* __restrict__ fx, int first, int n, int chunk,
              const int4* __restrict__ mlist, int K, double scale,
              unsigned long long* __restrict__ rho_fx) {
    __shared__ uint4 sp[kStage];
    const int l = blockIdx.y * kLTile + threadIdx.x;
    const bool active = l < K;
    const int4 m = active ? mlist[l] : make_int4(0, 0, 0, 0);
    const uint32_t mx = (uint32_t)m.x, my = (uint32_t)m.y, mz = (uint32_t)m.z;
    const int b0 = blockIdx.x * chunk;
    const int cnt_all = min(chunk, n - b0);
    float re = 0.f, im = 0.f;
    for (int base = 0; base < cnt_all; base += kStage) {
        const int cnt = min(kStage, cnt_all - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) sp[t] = fx[first + b0 + base + t];
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const uint4 p = sp[j];
                const uint32_t ph = mx * p.x + my * p.y + mz * p.z;
                float sn, cs;
                __sincosf((float)(int32_t)ph * kTwoPiOver2p32, &sn, &cs);
                const float q = __uint_as_float(p.w);
                re = fmaf(q, cs, re);
                im = fmaf(q, sn, im);
            }
        }
    }
    if (active && cnt_all > 0) rho_accumulate(rho_fx + 2 * l, (double)re, (double)im, scale);
}

// Energy and virial terms of the full structure factors, one thread per wave
// vector, FP64, summed per block in a fixed order: part[b] = (sum e_k, sum w_k)
// with e_k = 2 A_k |rho_k|^2 (half space: each k stands for +-k),
// A_k = (2 pi lB / V) e^{-k^2/(4 alpha)} / k^2, w_k = e_k (1 - k^2 / (2 alpha)).
__global__ void __launch_bounds__(256)
k_obs_terms(const __grid_constant__ SysDev S, const int4* __restrict__ mlist, int K,
            const unsigned long long* __restrict__ rho_fx, double2* __restrict__ part) {
    __shared__ double sa[256], sb[256];
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, wv = 0.0;
    if (l < K) {
        const double tp = 2.0 * M_PI * S.invL;
        const int4 m = mlist[l];
        const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
        const double2 r = rho_read(rho_fx + 2 * l, S.rho_inv_scale);
        e = 2.0 * (2.0 * M_PI * S.lB / S.V) * exp(-k2 / (4.0 * S.alpha)) / k2 *
            (r.x * r.x + r.y * r.y);
        wv = e * (1.0 - k2 / (2.0 * S.alpha));
    }
    sa[threadIdx.x] = e;
    sb[threadIdx.x] = wv;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sa[threadIdx.x] += sa[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sa[0], sb[0]);
}

// One block: the true energy and the virial of one system from the per-block
// wave-vector partials, the real-space Coulomb / LJ energies and virials of the
// preceding evaluation, the charges and the velocities, all summed in FP64 in
// a fixed order.  out[12]: E_total, E_fourier (incl. self and background),
// E_real, E_lj, E_kin, W_fourier, W_real, W_lj, W_background, pressure,
// kinetic temperature, 0.  P = (2 E_kin + W) / (3 V); W_bg = 3 E_bg.
__global__ void __launch_bounds__(256)
k_observables(const __grid_constant__ SysDev S, const double2* __restrict__ part, int nparts,
              const float4* __restrict__ pos_q, const float4* __restrict__ vel, int n,
              const double* __restrict__ E_in, const double* __restrict__ W_in, double mass,
              double* __restrict__ out) {
    __shared__ double sa[256], sb[256], sc[256], sd[256], se[256];
    double ef = 0.0, wf = 0.0, q1 = 0.0, q2 = 0.0, ke = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const double2 v = part[b];
        ef += v.x;
        wf += v.y;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double q = (double)pos_q[i].w;
        q1 += q;
        q2 += q * q;
        if (vel) {
            const float4 v = vel[i];
            ke += 0.5 * mass * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        }
    }
    sa[threadIdx.x] = ef; sb[threadIdx.x] = wf; sc[threadIdx.x] = q1; sd[threadIdx.x] = q2;
    se[threadIdx.x] = ke;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sa[threadIdx.x] += sa[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
            sd[threadIdx.x] += sd[threadIdx.x + o];
            se[threadIdx.x] += se[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ebg = -S.lB * M_PI * sc[0] * sc[0] / (2.0 * S.V * S.alpha);
        const double eself = -S.self_coef * sd[0];
        const double Ef = sa[0] + eself + ebg;
        const double Er = E_in[2], El = E_in[3];
        const double W = sb[0] + W_in[0] + W_in[1] + 3.0 * ebg;
        out[0] = Ef + Er + El;
        out[1] = Ef;
        out[2] = Er;
        out[3] = El;
        out[4] = se[0];
        out[5] = sb[0];
        out[6] = W_in[0];
        out[7] = W_in[1];
        out[8] = 3.0 * ebg;
        out[9] = (2.0 * se[0] + W) / (3.0 * S.V);
        out[10] = n > 0 ? 2.0 * se[0] / (3.0 * (double)n) : 0.0;
        out[11] = 0.0;
    }
}

void launch_observables(cudaStream_t st, const SysDev& S, const uint4* fx, int first, int n,
                        const int4* mlist, int K, unsigned long long* rho_fx, double2* part,
                        const float4* pos_q, const float4* vel, const double* E_in,
                        const double* W_in, double mass, double* out) {
    const int nparts = (K + 255) / 256;
    if (K > 0) {
        const int chunk = 1024;
        const int nch = std::max(1, (n + chunk - 1) / chunk);
        dim3 grid(nch, (K + kLTile - 1) / kLTile);
        cudaMemsetAsync(rho_fx, 0, sizeof(unsigned long long) * 2 * (size_t)K, st);
        if (n > 0)
            k_struct_full<<<grid, kLTile, 0, st>>>(fx, first, n, chunk, mlist, K, S.rho_scale,
                                                   rho_fx);
        k_obs_terms<<<nparts, 256, 0, st>>>(S, mlist, K, rho_fx, part);
    }
    k_observables<<<1, 256, 0, st>>>(S, part, nparts, pos_q + first,
                                     vel ? vel + first : nullptr, n, E_in, W_in, mass, out);
}

}  // namespace rbe
