// rbe_fused.cu -- one neighbour-list MD step of a single system (mixed path,
// exact k-sampler) in one cooperative launch.
//
// For systems of a few thousand particles every kernel of the multi-kernel
// step is latency-bound: a few hundred blocks each waiting on a handful of
// memory round trips, so the step costs mostly launch and drain latency.
// Here one persistent grid (every block resident, guaranteed by the
// cooperative launch) runs the step's phases back to back, separated by grid
// barriers:
//
//   A  prep: fixed-point records, displacement test against the last list
//      build, sorted records, the k-batch (Eq. probexpression), Nose-Hoover
//      friction, zeroed structure-factor accumulators
//   B  (only when some particle moved more than skin/2) cell counts, scan,
//      scatter, canonical order, list build -- five more barriers
//   C  structure-factor partials (Sec. 2, rho(k) in 64-bit fixed point) and
//      the real-space pass over the list, as independent work items
//   E  force coefficients of Eq. rbmapprox from rho(k), the Fourier force,
//      the total force and the thermostat update
//
// The arithmetic of every phase is that of the multi-kernel step (the same
// helpers and the same order within a particle's sums); only the scheduling
// differs.  The grid barrier spins on a generation word with a bounded number
// of waits: on timeout it latches kErrTimeout and the kernel returns.
#include <cmath>

#include "rbe_internal.cuh"

namespace rbe {

constexpr int kFT = 256;                 // threads per block
constexpr int kFStage = 512;             // particles staged per structure-factor pass
constexpr int kFMaxP = kFusedMaxP;       // wave vectors held in shared memory
constexpr unsigned kBarrierSpins = 4000000u;

// Grid barrier.  Thread 0 of each block reads the generation, arrives on the
// counter (after a fence that publishes the block's writes; the counter wraps
// to zero on the last arrival) and waits for the last arrival to advance the
// generation.  Returns false on timeout (all threads of the block agree); the
// host then clears the counter when it reports the timeout.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicInc(bar, gridDim.x - 1) == gridDim.x - 1) {
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned spins = 0;
            while (*gen == g) {
                if (++spins > kBarrierSpins) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------ phase A
__device__ void fused_prep(const FusedArgs& a, uint64_t step, uint32_t* s_tab) {
    const SysDev& S = a.S;
    const int t = threadIdx.x;
    if (blockIdx.x == 0 && t == 0) {
        *a.cur_step = step;
        if (a.nh && S.thermostat == RBE_THERMO_NOSE_HOOVER) {
            NhState st = a.nh[0];
            if (!st.first) st.xi += S.nh_rate * ((double)st.k2 * 0x1p-32 - 3.0 * (double)S.n);
            st.first = 0;
            st.k2 = 0ull;
            const double hx = 0.5 * st.xi * S.dt;
            st.a = 1.0 - hx;
            st.b = 1.0 / (1.0 + hx);
            st.f_va = (float)(st.a * st.b);
            st.f_vf = (float)(S.dt_over_m * st.b);
            a.nh[0] = st;
        }
    }
    for (int k = blockIdx.x * kFT + t; k < 2 * S.P; k += gridDim.x * kFT) a.rho_fx[k] = 0ull;
    int moved = 0;
    const float Lu = S.L_over_2_32;
    for (int i = blockIdx.x * kFT + t; i < a.n; i += gridDim.x * kFT) {
        const int si = __ldg(a.iperm + i);
        const uint4 r0 = __ldg(a.sref + i);
        const float4 p = a.pos[i];
        const uint4 rec = make_uint4(to_fixed(p.x, S.fx_hi, S.fx_lo), to_fixed(p.y, S.fx_hi, S.fx_lo),
                                     to_fixed(p.z, S.fx_hi, S.fx_lo), __float_as_uint(p.w));
        a.fx[i] = rec;
        const float dx = (float)(int32_t)(rec.x - r0.x) * Lu;
        const float dy = (float)(int32_t)(rec.y - r0.y) * Lu;
        const float dz = (float)(int32_t)(rec.z - r0.z) * Lu;
        moved |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > S.f_half_skin2;
        a.spos[si] = rec;
    }
    if (__syncthreads_or(moved) && t == 0) atomicOr(a.list_flag, 1);
    // the k-batch: the first ceil(P / kFT) blocks, tables staged in shared memory
    if (blockIdx.x * kFT < S.P) {
        if (a.tab_words > 0) {
            for (int j = t; j < a.tab_words; j += kFT) s_tab[j] = (uint32_t)__ldg(a.table + j);
            __syncthreads();
        }
        const int l = blockIdx.x * kFT + t;
        if (l < S.P)
            a.ksamp[l] = a.tab_words > 0 ? sample_one_smem(S, s_tab + S.off_t, l, step, a.err)
                                         : sample_one(S, a.table + S.off_t, l, step, a.err);
    }
}

// ------------------------------------------------------------------ phase B
__device__ void fused_count(const FusedArgs& a) {
    const SysDev& S = a.S;
    const int ncd = S.ncd;
    for (int i = blockIdx.x * kFT + threadIdx.x; i < a.n; i += gridDim.x * kFT) {
        const uint4 r = a.fx[i];
        const int c = (cell_of_fixed(r.z, ncd) * ncd + cell_of_fixed(r.y, ncd)) * ncd +
                      cell_of_fixed(r.x, ncd);
        a.cid[i] = c;
        a.rank[i] = atomicAdd(a.cell_cnt + c, 1);
    }
}

// exclusive scan of the cell counts by block 0, which also zeroes them
__device__ void fused_scan(const FusedArgs& a) {
    if (blockIdx.x != 0) return;
    __shared__ int warp_tot[kFT / 32];
    __shared__ int carry_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < a.ncell; base += kFT * 4) {
        const int i0 = base + t * 4;
        int v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < a.ncell) ? a.cell_cnt[i0 + k] : 0;
            sum += v[k];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int tv = lane < kFT / 32 ? warp_tot[lane] : 0;
            int ti = tv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += y;
            }
            if (lane < kFT / 32) warp_tot[lane] = ti - tv;
        }
        __syncthreads();
        int run = carry_s + warp_tot[w] + (incl - sum);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < a.ncell) {
                a.cell_start[i0 + k] = run;
                a.cell_cnt[i0 + k] = 0;
            }
            run += v[k];
        }
        __syncthreads();
        if (t == kFT - 1) carry_s = run;
        __syncthreads();
    }
    if (t == 0) a.cell_start[a.ncell] = carry_s;
}

__device__ void fused_scatter(const FusedArgs& a) {
    for (int i = blockIdx.x * kFT + threadIdx.x; i < a.n; i += gridDim.x * kFT)
        a.perm_tmp[a.cell_start[a.cid[i]] + a.rank[i]] = i;
}

// canonical order inside each cell: ascending fixed-point x, ties by index
__device__ void fused_order(const FusedArgs& a) {
    for (int s = blockIdx.x * kFT + threadIdx.x; s < a.n; s += gridDim.x * kFT) {
        const int i = a.perm_tmp[s];
        const int c = a.cid[i];
        const int b = a.cell_start[c], e = a.cell_start[c + 1];
        const uint32_t xi = a.fx[i].x;
        int r = 0;
        for (int k = b; k < e; ++k) {
            const int j = a.perm_tmp[k];
            const uint32_t xj = a.fx[j].x;
            r += (xj < xi || (xj == xi && j < i)) ? 1 : 0;
        }
        const int dst = b + r;
        a.perm[dst] = i;
        a.iperm[i] = dst;
        a.spos[dst] = a.fx[i];
    }
}

// the list: pairs within r_c + skin over the 27 cells, those within r_c first
__device__ void fused_build(const FusedArgs& a) {
    const SysDev& S = a.S;
    const int ncd = S.ncd;
    const float Lu = S.L_over_2_32, cut2 = S.f_list_cut2, rc2 = S.f_rc2;
    const int dlo = ncd < 3 ? 0 : -1, dhi = ncd < 3 ? 0 : 1;
    const size_t stride = (size_t)a.nbr_stride;
    unsigned most = 0;
    for (int i = blockIdx.x * kFT + threadIdx.x; i < a.n; i += gridDim.x * kFT) {
        const uint4 si = a.spos[i];
        const int cx = cell_of_fixed(si.x, ncd), cy = cell_of_fixed(si.y, ncd),
                  cz = cell_of_fixed(si.z, ncd);
        int* out = a.nbr + i;
        int n_in = 0, n_sk = 0;
        for (int dz = dlo; dz <= dhi; ++dz)
            for (int dy = dlo; dy <= dhi; ++dy) {
                const int zz = wrapc(cz + dz, ncd), yy = wrapc(cy + dy, ncd);
                int r0, e0, r1, e1;
                row_ranges(a.cell_start, (zz * ncd + yy) * ncd, cx, ncd, r0, e0, r1, e1);
                for (int part = 0; part < 2; ++part) {
                    const int b = part ? r1 : r0, e = part ? e1 : e0;
                    for (int j = b; j < e; ++j) {
                        const uint4 sj = a.spos[j];
                        const float dx = (float)(int32_t)(sj.x - si.x) * Lu;
                        const float dyy = (float)(int32_t)(sj.y - si.y) * Lu;
                        const float dzz = (float)(int32_t)(sj.z - si.z) * Lu;
                        const float r2 = fmaf(dx, dx, fmaf(dyy, dyy, dzz * dzz));
                        if (r2 < cut2 && j != i) {
                            if (n_in + n_sk < a.nbr_cap) {
                                const int slot = r2 < rc2 ? n_in : a.nbr_cap - 1 - n_sk;
                                out[(size_t)slot * stride] = j;
                            }
                            if (r2 < rc2) ++n_in; else ++n_sk;
                        }
                    }
                }
            }
        const int cnt = n_in + n_sk;
        if (cnt <= a.nbr_cap)
            for (int k = 0; k < n_sk; ++k)
                out[(size_t)(n_in + k) * stride] = out[(size_t)(a.nbr_cap - n_sk + k) * stride];
        a.ncnt[i] = min(cnt, a.nbr_cap);
        a.sref[a.perm[i]] = si;
        if (cnt > a.nbr_cap) atomicOr(a.err, kErrList);
        most = max(most, (unsigned)cnt);
    }
    const unsigned wmax = __reduce_max_sync(0xffffffffu, most);
    if ((threadIdx.x & 31) == 0 && wmax) atomicMax(a.list_stats + 1, (unsigned long long)wmax);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.list_stats, 1ull);
}

// ------------------------------------------------------------------ phase C
// structure-factor partials of one (chunk, wave-vector tile) item: two
// threads per wave vector, FP32 over a staged pass, FP64 beyond
__device__ void fused_rho_item(const FusedArgs& a, int chunk, int tile, uint4* sp,
                               double2* s_half) {
    const SysDev& S = a.S;
    const int half = threadIdx.x / kLTile;
    const int l = tile * kLTile + (threadIdx.x - half * kLTile);
    const bool active = l < S.P;
    const int first = chunk * a.rchunk;
    const int count = min(a.rchunk, a.n - first);
    int4 m = make_int4(0, 0, 0, 0);
    if (active) m = a.ksamp[l];
    const uint32_t mx = (uint32_t)m.x, my = (uint32_t)m.y, mz = (uint32_t)m.z;
    double red = 0.0, imd = 0.0;
    for (int base = 0; base < count; base += kFStage) {
        const int cnt = min(kFStage, count - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += kFT) sp[t] = a.fx[first + base + t];
        __syncthreads();
        float re = 0.f, im = 0.f;
        if (active) {
#pragma unroll 4
            for (int j = half; j < cnt; j += 2) {
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
        red += (double)re;
        imd += (double)im;
    }
    __syncthreads();
    if (half == 1) s_half[threadIdx.x - kLTile] = make_double2(red, imd);
    __syncthreads();
    if (half == 0 && active) {
        const double2 o = s_half[threadIdx.x];
        rho_accumulate(a.rho_fx + 2 * l, red + o.x, imd + o.y, S.rho_scale);
    }
}

// the real-space pass over the list for one tile of kFT / R particles
template <int R>
__device__ void fused_list_item(const FusedArgs& a, int item, float4* s_f) {
    constexpr int T = kFT / R;
    const SysDev& S = a.S;
    const int first = item * T;
    const int count = min(T, a.n - first);
    const int p = threadIdx.x / R, l = threadIdx.x - p * R;
    PairConst kc;
    kc.rc2 = S.f_rc2;
    kc.lj_rc2 = S.lj_eps != 0.0 ? S.f_lj_rc2 : 0.f;
    kc.alpha = S.f_alpha;
    kc.sa = S.f_sqrt_alpha;
    kc.two_sa_spi = S.f_two_sa_spi;
    kc.lB = S.f_lB;
    kc.lj_s2 = S.f_lj_sigma2;
    kc.lj_eps = S.f_lj_eps;
    kc.lj_shift = S.f_lj_shift;
    kc.vir = false;
    PairAcc acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (p < count) {
        const int i = first + p;
        const uint4 si = a.spos[i];
        const float lbqi = kc.lB * __uint_as_float(si.w);
        const float Lu = S.L_over_2_32;
        const int* nb = a.nbr + i;
        const size_t st = (size_t)a.nbr_stride;
        const int cnt = __ldcs(a.ncnt + i);
        constexpr int U = 8;
        int j[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int kk = l + q * R;
            j[q] = kk < a.nbr_cap ? __ldcs(nb + (size_t)kk * st) : 0;
        }
        for (int k0 = l;;) {
            uint4 sj[U];
#pragma unroll
            for (int q = 0; q < U; ++q) sj[q] = a.spos[j[q]];
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (k0 + q * R < cnt) pair_fixed(si, sj[q], Lu, lbqi, kc, acc);
            k0 += U * R;
            if (k0 >= cnt) break;
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int kk = k0 + q * R;
                j[q] = kk < cnt ? __ldcs(nb + (size_t)kk * st) : 0;
            }
        }
    }
    float fx = acc.fx, fy = acc.fy, fz = acc.fz;
#pragma unroll
    for (int o = R / 2; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o, R);
        fy += __shfl_down_sync(0xffffffffu, fy, o, R);
        fz += __shfl_down_sync(0xffffffffu, fz, o, R);
    }
    __syncthreads();                                   // s_f reused across items
    if (p < count && l == 0) s_f[p] = make_float4(fx, fy, fz, 0.f);
    __syncthreads();
    if ((int)threadIdx.x < count)
        a.freal[a.perm[first + threadIdx.x]] = s_f[threadIdx.x];
}

// ------------------------------------------------------------------ phase E
// the Fourier force of one tile of kFT / SPLIT particles from the block's
// coefficient tables, the total force and the thermostat update
template <int SPLIT>
__device__ void fused_force_item(const FusedArgs& a, int item, uint64_t step, const KPhase* kp,
                                 const KForce* kf, const float* kb, float4* s_t) {
    constexpr int TILE = kFT / SPLIT;
    const SysDev& S = a.S;
    const int first = item * TILE;
    const int count = min(TILE, a.n - first);
    const int sub = threadIdx.x % SPLIT, t = threadIdx.x / SPLIT;
    const bool nhm = a.nh && S.thermostat == RBE_THERMO_NOSE_HOOVER;
    // the closing update's inputs and the thermostat's noise, before the loop
    float4 e_fr = make_float4(0.f, 0.f, 0.f, 0.f), e_v = e_fr, e_r = e_fr;
    MdNoise e_z{0.f, 0.f, 0.f, false};
    const int te = threadIdx.x;
    if (te < count) {
        const int o = first + te;
        e_fr = a.freal[o];
        e_v = a.md_vel[o];
        e_r = a.md_pos[o];
        if (!nhm) e_z = md_noise(S, step, o);
    }
    const uint4 p = a.fx[first + min(t, count - 1)];
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll 4
    for (int k = sub; k < S.P; k += SPLIT) {
        const KPhase kpk = kp[k];
        const uint32_t phs = kpk.mx * p.x + kpk.my * p.y + kpk.mz * p.z;
        const float th = (float)(int32_t)phs * kTwoPiOver2p32;
        float sn, cs;
        __sincosf(th, &sn, &cs);
        const KForce f = kf[k];
        const float g = fmaf(cs, f.A, -sn * kb[k]);      // Im(e^{-i th} rho) * coef
        fx = fmaf(g, f.mx, fx);
        fy = fmaf(g, f.my, fy);
        fz = fmaf(g, f.mz, fz);
    }
#pragma unroll
    for (int o = SPLIT / 2; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o, SPLIT);
        fy += __shfl_down_sync(0xffffffffu, fy, o, SPLIT);
        fz += __shfl_down_sync(0xffffffffu, fz, o, SPLIT);
    }
    __syncthreads();                                   // s_t reused across items
    if (t < count && sub == 0) {
        const float sc = -__uint_as_float(p.w) * (float)(2.0 * M_PI) * S.f_invL;
        s_t[t] = make_float4(sc * fx, sc * fy, sc * fz, 0.f);
    }
    __syncthreads();
    unsigned long long k2 = 0ull;
    if (te < count) {
        const int o = first + te;
        const float4 ff = s_t[te];
        const float Fx = e_fr.x + ff.x, Fy = e_fr.y + ff.y, Fz = e_fr.z + ff.z;
        if (a.F_out) a.F_out[o] = make_float4(Fx, Fy, Fz, 0.f);
        if (nhm)
            k2 = nose_hoover_apply(S, a.nh[0].f_va, a.nh[0].f_vf, Fx, Fy, Fz, e_v, e_r);
        else
            md_apply(S, e_z, Fx, Fy, Fz, e_v, e_r);
        a.md_vel[o] = e_v;
        a.md_pos[o] = e_r;
    }
    if (nhm) warp_add_u64(k2, &a.nh[0].k2);
}

// ------------------------------------------------------------------ kernel
template <int R, int SPLIT>
__global__ void __launch_bounds__(kFT) k_fused_step(const __grid_constant__ FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SysDev& S = a.S;
    const uint64_t step = a.step_dev ? *a.step_dev : a.step_arg;
    // A
    fused_prep(a, step, (uint32_t*)smem);
    if (!grid_barrier(a.bar, a.err)) return;
    // B: a rebuild when some particle moved beyond skin/2
    if (*(volatile int*)a.list_flag) {
        fused_count(a);
        if (!grid_barrier(a.bar, a.err)) return;
        fused_scan(a);
        if (!grid_barrier(a.bar, a.err)) return;
        fused_scatter(a);
        if (!grid_barrier(a.bar, a.err)) return;
        fused_order(a);
        if (!grid_barrier(a.bar, a.err)) return;
        fused_build(a);
        if (!grid_barrier(a.bar, a.err)) return;
    }
    // C: structure-factor items, then list items
    {
        uint4* sp = (uint4*)smem;                                   // [kFStage]
        double2* s_half = (double2*)(sp + kFStage);                 // [kLTile]
        float4* s_f = (float4*)(s_half + kLTile);                   // [kFT / R]
        const int nchunk = (a.n + a.rchunk - 1) / a.rchunk;
        const int ntile = (S.P + kLTile - 1) / kLTile;
        const int nrho = nchunk * ntile;
        const int nlist = (a.n + kFT / R - 1) / (kFT / R);
        for (int it = blockIdx.x; it < nrho + nlist; it += gridDim.x) {
            if (it < nrho) fused_rho_item(a, it / ntile, it % ntile, sp, s_half);
            else fused_list_item<R>(a, it - nrho, s_f);
        }
    }
    if (!grid_barrier(a.bar, a.err)) return;
    // E: coefficient tables in shared memory, then the force items
    {
        KPhase* kp = (KPhase*)smem;                                 // [P]
        KForce* kf = (KForce*)(kp + kFMaxP);                        // [P]
        float* kb = (float*)(kf + kFMaxP);                          // [P]
        float4* s_t = (float4*)(kb + kFMaxP);                       // [kFT / SPLIT]
        const double tp = 2.0 * M_PI * S.invL;
        for (int l = threadIdx.x; l < S.P; l += kFT) {
            const int4 m = a.ksamp[l];
            const double2 r = rho_read(a.rho_fx + 2 * l, S.rho_inv_scale);
            const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
            const double c = S.coef_scale / k2;
            kp[l] = KPhase{(uint32_t)m.x, (uint32_t)m.y, (uint32_t)m.z, 0u};
            kf[l] = KForce{(float)m.x, (float)m.y, (float)m.z, (float)(c * r.y)};
            kb[l] = (float)(c * r.x);
        }
        __syncthreads();
        const int nforce = (a.n + kFT / SPLIT - 1) / (kFT / SPLIT);
        for (int it = blockIdx.x; it < nforce; it += gridDim.x)
            fused_force_item<SPLIT>(a, it, step, kp, kf, kb, s_t);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.list_flag = 0;                              // this step's rebuild is done
        if (a.step_dev) *a.step_dev = step + 1;
    }
}

// Shared memory of the kernel: the largest of the phases' needs.
static size_t fused_smem(int tab_words) {
    const size_t a_ = sizeof(uint32_t) * (size_t)tab_words;
    const size_t c_ = sizeof(uint4) * kFStage + sizeof(double2) * kLTile + sizeof(float4) * kFT;
    const size_t e_ = (sizeof(KPhase) + sizeof(KForce) + sizeof(float)) * kFMaxP +
                      sizeof(float4) * kFT;
    return std::max(a_, std::max(c_, e_));
}

template <int R, int SPLIT>
static cudaError_t fused_launch(cudaStream_t st, const FusedArgs& a, int grid) {
    const size_t smem = fused_smem(a.tab_words);
    cudaError_t e = cudaFuncSetAttribute(k_fused_step<R, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kFT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fused_step<R, SPLIT>, a);
}

// Blocks the cooperative grid may hold on this device (resident at once),
// capped at two per SM; 0 if cooperative launches are not available.
template <int R, int SPLIT>
static int fused_grid_rs(int tab_words) {
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = fused_smem(tab_words);
    if (cudaFuncSetAttribute(k_fused_step<R, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_step<R, SPLIT>, kFT, smem) !=
        cudaSuccess)
        return 0;
    if (!coop || per_sm < 1) return 0;
    return sms * std::min(per_sm, 2);
}

int fused_grid(const FusedArgs& a) {
#define RBE_G(R, S) fused_grid_rs<R, S>(a.tab_words)
    switch (a.rsplit * 16 + a.fsplit) {
        case 8 * 16 + 8: return RBE_G(8, 8);
        case 8 * 16 + 4: return RBE_G(8, 4);
        case 4 * 16 + 8: return RBE_G(4, 8);
        case 4 * 16 + 4: return RBE_G(4, 4);
        case 2 * 16 + 4: return RBE_G(2, 4);
        case 2 * 16 + 2: return RBE_G(2, 2);
        case 1 * 16 + 2: return RBE_G(1, 2);
        default: return RBE_G(1, 1);
    }
#undef RBE_G
}

cudaError_t launch_fused_step(cudaStream_t st, const FusedArgs& a, int grid) {
    switch (a.rsplit * 16 + a.fsplit) {
        case 8 * 16 + 8: return fused_launch<8, 8>(st, a, grid);
        case 8 * 16 + 4: return fused_launch<8, 4>(st, a, grid);
        case 4 * 16 + 8: return fused_launch<4, 8>(st, a, grid);
        case 4 * 16 + 4: return fused_launch<4, 4>(st, a, grid);
        case 2 * 16 + 4: return fused_launch<2, 4>(st, a, grid);
        case 2 * 16 + 2: return fused_launch<2, 2>(st, a, grid);
        case 1 * 16 + 2: return fused_launch<1, 2>(st, a, grid);
        default: return fused_launch<1, 1>(st, a, grid);
    }
}

}  // namespace rbe
