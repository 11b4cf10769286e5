// rbe_cells.cu -- per-step preparation: fixed-point fractional coordinates,
// cell assignment and a counting sort of the particles by cell.
//
// The real-space sum of Eq. force (second term) needs every pair closer than
// r_c.  Cells of side >= r_c + skin (n_cells_dim = floor(L / (r_c + skin)) >= 3
// per edge, skin 0 without a neighbour list) make that a walk over the 27
// neighbouring cells, and the neighbour list of the MD step a walk over the
// same cells with the cutoff r_c + skin.  The sort is a counting sort
// (histogram with atomics, one exclusive scan, scatter), followed by a per-cell
// re-ordering by original index so that the order inside a cell -- and with it
// every floating-point sum over neighbours -- is the same on every run.
//
// Mixed path: a coordinate x is stored as the 32-bit fixed-point fraction
// round(2^32 x / L) mod 2^32.  The product 2^32 x / L is formed exactly enough
// in FP32 by splitting 2^32 / L into a float pair (hi + lo) and recovering the
// rounding error of x * hi with an FMA, so the stored fraction is within one
// unit (L / 2^32) of the exact one for any float x.  Periodic wrapping is then
// the natural 2^32 modulus, m . s mod 1 is exact in integer arithmetic, and
// the minimum-image displacement is the signed difference of two fractions.
#include "rbe_internal.cuh"

namespace rbe {

// FP32 and 32-bit integer work only (64-bit conversions would go through the
// FP64 pipe, which is narrow on this part): the integer pr is first reduced
// modulo 2^32 in FP32, exactly, to r in [-2^31, 2^31] (for |pr| >= 2^31 the
// result is a multiple of ulp(pr) >= 2^8 below 2^31 in magnitude, so it is a
// float; below that pr is left as it is).  Same fraction as the 64-bit sum
// ip + ic mod 2^32 for |x| < 2^31 L.
__device__ __forceinline__ uint32_t to_fixed(float x, float hi, float lo) {
    const float p = x * hi;
    const float e = fmaf(x, hi, -p);       // exact: x * hi = p + e
    float corr = fmaf(x, lo, e);
    const float pr = rintf(p);
    corr += (p - pr);                      // exact (p and pr differ by < 1 ulp-scale)
    const float n = rintf(pr * 2.3283064365386963e-10f);        // pr / 2^32, nearest
    const float r = fmaf(-4294967296.0f, n, pr);                 // exact, |r| <= 2^31
    // 2^31 and -2^31 are the same fraction; the conversion saturates at 2^31 - 1
    const uint32_t ur = r >= 2147483648.0f ? 0x80000000u : (uint32_t)__float2int_rz(r);
    return ur + (uint32_t)__float2int_rn(corr);
}

__device__ __forceinline__ int cell_of_fixed(uint32_t s, int ncd) {
    return (int)(((unsigned long long)s * (unsigned long long)ncd) >> 32);
}

// Deterministic block sum of two doubles (fixed shuffle tree, then warps in order).
__device__ __forceinline__ double2 block_sum2(double a, double b) {
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

// Thread 0 of block 0 latches the step index of this evaluation: the
// caller's device counter or the host value.  The counter is advanced by the
// cell-count scan, a later kernel, so every block of this one reads the same
// value.
__device__ __forceinline__ void latch_step(const uint64_t* step_dev, uint64_t step_arg,
                                          uint64_t* cur_step, int pb) {
    if (pb == 0 && threadIdx.x == 0) *cur_step = step_dev ? *step_dev : step_arg;
}

// Nose-Hoover (the equations of motion of Sec. 3.3): thread s of block 0
// advances the friction of system s from the kinetic sum of the previous step,
// xi += dt / Q (sum m|v|^2 - 3 n kT) with Q = 3 n kT tau^2 (not on the first
// step after a reset), and sets this step's velocity coefficients.  The
// real-space kernel of this step, launched after this one, reads them and
// accumulates the next sum.
template <bool ONE>
__device__ __forceinline__ void nh_advance(const Work& w, const PrepArgs& pa, int pb) {
    if (!pa.nh || pb != 0) return;
    for (int s = threadIdx.x; s < pa.nsys; s += blockDim.x) {
        const SysDev& S = sys_of<ONE>(w, s);
        if (S.thermostat != RBE_THERMO_NOSE_HOOVER) continue;
        NhState st = pa.nh[s];
        if (!st.first) st.xi += S.nh_rate * ((double)st.k2 * 0x1p-32 - 3.0 * (double)S.n);
        st.first = 0;
        st.k2 = 0ull;
        const double hx = 0.5 * st.xi * S.dt;
        st.a = 1.0 - hx;
        st.b = 1.0 / (1.0 + hx);
        st.f_va = (float)(st.a * st.b);
        st.f_vf = (float)(S.dt_over_m * st.b);
        pa.nh[s] = st;
    }
}

// The k-batch of this step (Eq. probexpression): the blocks before the particle
// blocks draw one sample per thread and its coefficient coef_scale / k^2 of
// Eq. rbmapprox, for the structure-factor and force passes that follow.
// The paper's Metropolis-Hastings sampler (Sec. 3.1), one block per system:
// three per-axis independence chains with the rounded-Gaussian proposal, run
// in windows of kMhWin iterations (one window covers P up to about 250).  Proposals and uniforms of a window come
// from Philox in parallel (iteration t, axis c: ctr = (t_lo, t_hi, c,
// (stream << 8) | 6)); threads 0..2 then walk their chain through the window
// (accept m* iff u * rho(m) < rho(m*)); thread 0 keeps the nonzero triples in
// order until P are out.  The chains' state and position persist in the handle
// (the set K of Algorithm 1, consumed in order).
constexpr int kMhWin = 256;

template <bool ONE>
__device__ void draw_samples_mh(const Work& w, const PrepArgs& pa, int sb) {
    extern __shared__ __align__(16) unsigned char mh_smem[];
    double* s_rho = (double*)mh_smem;                          // [mh_words]
    uint32_t* s_tq = (uint32_t*)(s_rho + pa.mh_words);         // [mh_words]
    __shared__ int s_prop[3][kMhWin];
    __shared__ double s_u[3][kMhWin];
    __shared__ unsigned char s_dec[3][kMhWin];   // decision if the state is the previous proposal
    __shared__ int s_st[3][kMhWin];
    __shared__ int s_state[3], s_emitted, s_used, s_bad;
    __shared__ int s_wsum[kBlockP / 32];
    static_assert(kMhWin == 2 * kBlockP, "emission takes two window iterations per thread");
    const int sys = sb;
    if (sys >= pa.nsys) return;
    const SysDev& S = sys_of<ONE>(w, sys);
    const int n = 2 * S.M + 1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        s_rho[j] = __ldg(pa.mh_rho + S.off_t + j);
        s_tq[j] = (uint32_t)__ldg(pa.mh_tq + S.off_t + j);   // entry 2M (= 2^32) is never read
    }
    if (threadIdx.x < 3) s_state[threadIdx.x] = (&pa.mh_state[sys].x)[threadIdx.x];
    if (threadIdx.x == 0) { s_emitted = 0; s_bad = 0; }
    __syncthreads();
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    uint64_t t0 = pa.mh_pos[sys];
    const uint64_t tmax = t0 + 64ull * (uint64_t)S.P + 1024ull;
    while (s_emitted < S.P && !s_bad) {
        for (int idx = threadIdx.x; idx < 3 * kMhWin; idx += blockDim.x) {
            const int c = idx / kMhWin, it = idx - c * kMhWin;
            const uint64_t t = t0 + (uint64_t)it;
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)c, (S.stream << 8) | 0x06u), key);
            int lo = 0, hi = n - 1;                 // smallest j with r.x < T[j] (T[n-1] = 2^32)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (r.x < s_tq[mid]) hi = mid; else lo = mid + 1;
            }
            s_prop[c][it] = lo - S.M;
            s_u[c][it] = (double)((((unsigned long long)r.z << 32) | r.w) >> 11) * 0x1.0p-53;
        }
        __syncthreads();
        // The acceptance test depends on the state only through its value, and the
        // state is nearly always the previous proposal: decide every iteration for
        // that state in parallel; the walk below recomputes only when it differs.
        for (int idx = threadIdx.x; idx < 3 * kMhWin; idx += blockDim.x) {
            const int c = idx / kMhWin, it = idx - c * kMhWin;
            if (it > 0)
                s_dec[c][it] = __dmul_rn(s_u[c][it], s_rho[s_prop[c][it - 1] + S.M]) <
                               s_rho[s_prop[c][it] + S.M];
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            // the walk: the state enters only through a compare and a select, so
            // the proposals and decisions of eight iterations are loaded at once
            const int c = threadIdx.x;
            int st = s_state[c];
            for (int it0 = 0; it0 < kMhWin; it0 += 8) {
                int pr[9];
                unsigned char dc[8];
                pr[0] = it0 > 0 ? s_prop[c][it0 - 1] : 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    pr[q + 1] = s_prop[c][it0 + q];
                    dc[q] = s_dec[c][it0 + q];
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int it = it0 + q, ms = pr[q + 1];
                    const bool acc = (it > 0 && st == pr[q])
                                         ? dc[q] != 0
                                         : __dmul_rn(s_u[c][it], s_rho[st + S.M]) < s_rho[ms + S.M];
                    if (acc) st = ms;
                    s_st[c][it] = st;
                }
            }
        }
        __syncthreads();
        // emission: the nonzero triples of the window in order, until P are out;
        // each finds its slot from a block-wide prefix count of the nonzero ones
        {
            const int e0 = s_emitted, need = S.P - e0;
            const int a0 = 2 * threadIdx.x, a1 = a0 + 1;          // kMhWin == 2 * kBlockP
            const bool f0 = (s_st[0][a0] | s_st[1][a0] | s_st[2][a0]) != 0;
            const bool f1 = (s_st[0][a1] | s_st[1][a1] | s_st[2][a1]) != 0;
            const int mine = (int)f0 + (int)f1;
            int incl = mine;
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[wid] = incl;
            if (threadIdx.x == 0) s_used = kMhWin;
            __syncthreads();
            int before = 0, total = 0;
            for (int k = 0; k < kBlockP / 32; ++k) {
                if (k < wid) before += s_wsum[k];
                total += s_wsum[k];
            }
            const int p0 = before + incl - mine;               // nonzero triples before a0
            if (f0 && p0 < need) {
                pa.ksamp[S.off_k + e0 + p0] = make_int4(s_st[0][a0], s_st[1][a0], s_st[2][a0], 1);
                if (p0 == need - 1) s_used = a0 + 1;
            }
            const int p1 = p0 + (int)f0;
            if (f1 && p1 < need) {
                pa.ksamp[S.off_k + e0 + p1] = make_int4(s_st[0][a1], s_st[1][a1], s_st[2][a1], 1);
                if (p1 == need - 1) s_used = a1 + 1;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const int used = s_used;
                const int e = min(e0 + total, S.P);
                for (int c = 0; c < 3; ++c) s_state[c] = s_st[c][used - 1];
                s_emitted = e;
                if (t0 + (uint64_t)used >= tmax && e < S.P) s_bad = 1;
            }
            __syncthreads();
        }
        t0 += (uint64_t)s_used;
    }
    if (threadIdx.x == 0) {
        pa.mh_state[sys] = make_int4(s_state[0], s_state[1], s_state[2], 0);
        pa.mh_pos[sys] = t0;
        if (s_bad) {
            atomicOr(pa.err, kErrSampler);
            for (int l = s_emitted; l < S.P; ++l) pa.ksamp[S.off_k + l] = make_int4(1, 0, 0, 0);
        }
    }
    __syncthreads();
    const double tp = 2.0 * M_PI * S.invL;
    for (int l = threadIdx.x; l < S.P; l += blockDim.x) {
        const int4 m = pa.ksamp[S.off_k + l];
        const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
        pa.kcoef[S.off_k + l] = S.coef_scale / k2;
    }
}

template <bool ONE>
__device__ __forceinline__ void draw_samples(const Work& w, const PrepArgs& pa, int sb) {
    extern __shared__ uint32_t s_tab[];
    if (pa.tab_words > 0) {
        for (int j = threadIdx.x; j < pa.tab_words; j += blockDim.x)
            s_tab[j] = (uint32_t)__ldg(pa.table + j);
        __syncthreads();
    }
    const int g = sb * blockDim.x + threadIdx.x;
    if (g >= pa.ktot) return;
    const int s = ONE ? 0 : find_sys(pa.kstart, pa.nsys, g);
    const SysDev& S = sys_of<ONE>(w, s);
    const uint64_t step = pa.step_dev ? *pa.step_dev : pa.step_arg;
    const int4 m = pa.tab_words > 0
                       ? sample_one_smem(S, s_tab + S.off_t, g - S.off_k, step, pa.err)
                       : sample_one(S, pa.table + S.off_t, g - S.off_k, step, pa.err);
    pa.ksamp[g] = m;
    const double tp = 2.0 * M_PI * S.invL;
    const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
    pa.kcoef[g] = S.coef_scale / k2;
}

// Zero the rho(k) accumulators for this evaluation (stride over the nblk
// particle blocks, pb the block's index among them; the sampling blocks do not
// take part).
__device__ __forceinline__ void clear_rho(unsigned long long* rho_fx, int nrho, int nblk, int pb) {
    for (int k = pb * blockDim.x + threadIdx.x; k < 2 * nrho; k += nblk * blockDim.x)
        rho_fx[k] = 0ull;
}

template <bool ONE>
__global__ void __launch_bounds__(kBlockP)
k_prep_mixed(const __grid_constant__ Work w, const float4* __restrict__ pos_q,
             uint4* __restrict__ fx, int* __restrict__ cid, int* __restrict__ rank,
             int* __restrict__ cell_cnt, const __grid_constant__ PrepArgs pa) {
    pdl_trigger();                     // a dependent kernel may be scheduled meanwhile
    // the k-sampling blocks come first, so that their table staging and
    // searches run alongside the particle blocks instead of after them
    const int nsb = (int)gridDim.x - pa.npblk;
    if ((int)blockIdx.x < nsb) {
        if (pa.mh) draw_samples_mh<ONE>(w, pa, (int)blockIdx.x);
        else draw_samples<ONE>(w, pa, (int)blockIdx.x);
        return;
    }
    const int pb = (int)blockIdx.x - nsb;          // this particle block
    latch_step(pa.step_dev, pa.step_arg, pa.cur_step, pb);
    nh_advance<ONE>(w, pa, pb);
    clear_rho(pa.rho_fx, pa.nrho, pa.npblk, pb);
    const Tile tl = tile_at<ONE>(w, pb);
    const SysDev& S = sys_of<ONE>(w, tl.sys);
    const int t = threadIdx.x;
    double qs = 0.0, q2s = 0.0;
    int moved = 0;
    if (t < tl.count) {
        const int i = tl.first + t;
        // list step: the sorted slot and the record of the last build, loaded
        // with the position
        const int si = pa.list_flag ? __ldg(pa.iperm + i) : 0;
        const uint4 r0 = pa.list_flag ? __ldg(pa.sref + i) : make_uint4(0, 0, 0, 0);
        const float4 p = pos_q[i];
        // a NaN or infinite input is latched (RBE_ERR_NONFINITE at the next
        // synchronisation); its fixed-point record is some 32-bit pattern, so
        // every index derived from it stays in range
        latch_any(!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w)), pa.err,
                  kErrNonfinite);
        const uint32_t sx = to_fixed(p.x, S.fx_hi, S.fx_lo);
        const uint32_t sy = to_fixed(p.y, S.fx_hi, S.fx_lo);
        const uint32_t sz = to_fixed(p.z, S.fx_hi, S.fx_lo);
        if (!pa.list_flag) {
            // the cell of the particle and its slot in the cell's count; a
            // neighbour-list evaluation leaves this to k_cell_assign, which
            // runs only when the list is rebuilt
            const int ncd = S.ncd;
            const int c = S.off_c +
                          (cell_of_fixed(sz, ncd) * ncd + cell_of_fixed(sy, ncd)) * ncd +
                          cell_of_fixed(sx, ncd);
            cid[i] = c;
            rank[i] = RBE_IN_BOUNDS(c, pa.ncell, pa.err) ? atomicAdd(cell_cnt + c, 1) : 0;
        }
        const uint4 rec = make_uint4(sx, sy, sz, __float_as_uint(p.w));
        fx[i] = rec;
        if (pa.want_q) {
            qs = (double)p.w;
            q2s = (double)p.w * (double)p.w;
        }
        if (pa.list_flag) {
            // neighbour-list step: the record goes to its sorted slot of the
            // last build, and a displacement beyond skin/2 since that build
            // (minimum image, from the fixed-point difference) asks for a new list
            const float Lu = S.L_over_2_32;
            const float dx = (float)(int32_t)(sx - r0.x) * Lu;
            const float dy = (float)(int32_t)(sy - r0.y) * Lu;
            const float dz = (float)(int32_t)(sz - r0.z) * Lu;
            moved = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > S.f_half_skin2;
            if (RBE_IN_BOUNDS(si, pa.ntot, pa.err)) pa.spos[si] = rec;
        }
    }
    if (pa.list_flag) {
        if (__syncthreads_or(moved) && t == 0) atomicOr(pa.list_flag, 1);
    }
    if (pa.want_q) {
        const double2 r = block_sum2(qs, q2s);
        if (t == 0) {
            pa.blk_q[pb] = r;
            atomicAdd(pa.qsum_fx + tl.sys, (unsigned long long)__double2ll_rn(r.x * kQScale));
        }
    }
}

__device__ __forceinline__ double wrap_f64(double x, double L, double invL) {
    double w = x - L * floor(x * invL);
    if (w >= L) w -= L;
    if (!(w >= 0.0)) w = 0.0;      // also maps NaN to 0
    return w;
}

__device__ __forceinline__ int cell_of_f64(double w, double invL, int ncd) {
    const double u = w * invL * (double)ncd;
    int c = (u >= 0.0 && u < (double)ncd) ? (int)u : 0;
    return c;
}

template <bool ONE>
__global__ void __launch_bounds__(kBlockP)
k_prep_f64(const __grid_constant__ Work w, const double4* __restrict__ pos_q,
           double4* __restrict__ fx64, int* __restrict__ cid, int* __restrict__ rank,
           int* __restrict__ cell_cnt, const __grid_constant__ PrepArgs pa) {
    // the k-sampling blocks come first, so that their table staging and
    // searches run alongside the particle blocks instead of after them
    const int nsb = (int)gridDim.x - pa.npblk;
    if ((int)blockIdx.x < nsb) {
        if (pa.mh) draw_samples_mh<ONE>(w, pa, (int)blockIdx.x);
        else draw_samples<ONE>(w, pa, (int)blockIdx.x);
        return;
    }
    const int pb = (int)blockIdx.x - nsb;          // this particle block
    latch_step(pa.step_dev, pa.step_arg, pa.cur_step, pb);
    nh_advance<ONE>(w, pa, pb);
    clear_rho(pa.rho_fx, pa.nrho, pa.npblk, pb);
    const Tile tl = tile_at<ONE>(w, pb);
    const SysDev& S = sys_of<ONE>(w, tl.sys);
    const int t = threadIdx.x;
    double qs = 0.0, q2s = 0.0;
    if (t < tl.count) {
        const int i = tl.first + t;
        const double4 p = pos_q[i];
        latch_any(!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w)), pa.err,
                  kErrNonfinite);
        const double x = wrap_f64(p.x, S.L, S.invL);
        const double y = wrap_f64(p.y, S.L, S.invL);
        const double z = wrap_f64(p.z, S.L, S.invL);
        const int ncd = S.ncd;
        const int c = S.off_c +
                      (cell_of_f64(z, S.invL, ncd) * ncd + cell_of_f64(y, S.invL, ncd)) * ncd +
                      cell_of_f64(x, S.invL, ncd);
        cid[i] = c;
        rank[i] = RBE_IN_BOUNDS(c, pa.ncell, pa.err) ? atomicAdd(cell_cnt + c, 1) : 0;
        fx64[i] = make_double4(x, y, z, p.w);
        qs = p.w;
        q2s = p.w * p.w;
    }
    if (pa.want_q) {
        const double2 r = block_sum2(qs, q2s);
        if (t == 0) {
            pa.blk_q[pb] = r;
            atomicAdd(pa.qsum_fx + tl.sys, (unsigned long long)__double2ll_rn(r.x * kQScale));
        }
    }
}

// Neighbour-list evaluations: the cells of the particles and their slots in
// the cell counts, from the fixed-point records of the prep kernel, only when
// this evaluation rebuilds the list (the prep kernel set the flag).
template <bool ONE>
__global__ void __launch_bounds__(kBlockP)
k_cell_assign(const __grid_constant__ Work w, const uint4* __restrict__ fx, int* __restrict__ cid,
              int* __restrict__ rank, int* __restrict__ cell_cnt, int ncell,
              const int* __restrict__ list_flag, int* __restrict__ err) {
    if (!*list_flag) return;
    const Tile tl = tile_of<ONE>(w);
    const SysDev& S = sys_of<ONE>(w, tl.sys);
    const int t = threadIdx.x;
    if (t >= tl.count) return;
    const int i = tl.first + t;
    const uint4 r = fx[i];
    const int ncd = S.ncd;
    const int c = S.off_c + (cell_of_fixed(r.z, ncd) * ncd + cell_of_fixed(r.y, ncd)) * ncd +
                  cell_of_fixed(r.x, ncd);
    cid[i] = c;
    rank[i] = RBE_IN_BOUNDS(c, ncell, err) ? atomicAdd(cell_cnt + c, 1) : 0;
}

// Exclusive scan of the cell counts (one block), zeroing the counts for the
// next call.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;

__global__ void __launch_bounds__(kScanThreads)
k_scan(int* __restrict__ cell_cnt, int* __restrict__ cell_start, int ncell,
       uint64_t* __restrict__ step_dev, const uint64_t* __restrict__ cur_step,
       const int* __restrict__ list_flag) {
    if (step_dev && threadIdx.x == 0) *step_dev = *cur_step + 1;   // one increment per step
    // the list stands: no cell was counted (k_cell_assign counts only for a
    // rebuild, and every scan leaves the counts at zero)
    if (list_flag && !*list_flag) return;
    __shared__ int warp_tot[kScanThreads / 32];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += kScanThreads * kScanPer) {
        const int i0 = base + threadIdx.x * kScanPer;
        int v[kScanPer];
        int sum = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = i0 + k;
            v[k] = (i < ncell) ? cell_cnt[i] : 0;
            sum += v[k];
        }
        // inclusive warp scan of per-thread sums
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        if (w == 0) {
            int t = warp_tot[lane];
            int ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += y;
            }
            warp_tot[lane] = ti - t;    // exclusive prefix of warp totals
        }
        __syncthreads();
        int run = carry_s + warp_tot[w] + (incl - sum);
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = i0 + k;
            if (i < ncell) {
                cell_start[i] = run;
                cell_cnt[i] = 0;
            }
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry_s = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) cell_start[ncell] = carry_s;
}

// Scatter of the caller's indices to their atomic slots (arbitrary order
// inside each cell).
__global__ void k_scatter(int n, const int* __restrict__ cid, const int* __restrict__ rank,
                          const int* __restrict__ cell_start, int* __restrict__ perm_tmp,
                          const int* __restrict__ list_flag, int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (list_flag && !*list_flag)) return;
    const int slot = cell_start[cid[i]] + rank[i];
    if (RBE_IN_BOUNDS(slot, n, err)) perm_tmp[slot] = i;
}

// Canonical order inside each cell: the particle at atomic slot s goes to
// cell_start + (number of members of its cell that precede it).  The mixed
// path orders by fixed-point x (ties by caller index), which the real-space
// kernel's x windows rely on; the FP64 path by caller index.  One thread per
// particle; cells hold a handful of particles.
__global__ void k_order(int n, const int* __restrict__ cid, const int* __restrict__ cell_start,
                        const int* __restrict__ perm_tmp, const uint4* __restrict__ fx,
                        uint4* __restrict__ spos, const double4* __restrict__ fx64,
                        double4* __restrict__ spos64, int* __restrict__ perm,
                        const int* __restrict__ list_flag, int* __restrict__ iperm,
                        int* __restrict__ err) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || (list_flag && !*list_flag)) return;
    const int i = perm_tmp[s];
    if (!RBE_IN_BOUNDS(i, n, err)) return;
    const int c = cid[i];
    const int b = cell_start[c], e = cell_start[c + 1];
    int r = 0;
    if (fx) {
        // mixed path: ascending fixed-point x, ties by index
        const uint32_t xi = fx[i].x;
        for (int k = b; k < e; ++k) {
            const int j = __ldg(perm_tmp + k);
            const uint32_t xj = __ldg(&fx[j].x);
            r += (xj < xi || (xj == xi && j < i)) ? 1 : 0;
        }
    } else {
        for (int k = b; k < e; ++k) r += (__ldg(perm_tmp + k) < i) ? 1 : 0;
    }
    const int dst = b + r;
    if (!RBE_IN_BOUNDS(dst, n, err)) return;
    perm[dst] = i;
    if (iperm) iperm[i] = dst;
    if (fx) spos[dst] = fx[i];
    if (fx64) spos64[dst] = fx64[i];
}

// ------------------------------------------------------------- launchers
void launch_prep_mixed(cudaStream_t st, bool one, const Work& w, int nblk, const float4* pos_q,
                       uint4* fx, int* cid, int* rank, int* cell_cnt, const PrepArgs& pa) {
    // particle blocks, then sampling blocks: one per system (MH chains) or one per kBlockP samples
    if (pa.ktot > 0) nblk += pa.mh ? pa.nsys : (pa.ktot + kBlockP - 1) / kBlockP;
    if (nblk <= 0) return;
    const size_t smem = pa.mh ? (sizeof(double) + sizeof(uint32_t)) * (size_t)pa.mh_words
                              : sizeof(uint32_t) * (size_t)pa.tab_words;
    if (one)
        k_prep_mixed<true><<<nblk, kBlockP, smem, st>>>(w, pos_q, fx, cid, rank, cell_cnt, pa);
    else
        k_prep_mixed<false><<<nblk, kBlockP, smem, st>>>(w, pos_q, fx, cid, rank, cell_cnt, pa);
}

void launch_prep_f64(cudaStream_t st, bool one, const Work& w, int nblk, const double4* pos_q,
                     double4* fx64, int* cid, int* rank, int* cell_cnt, const PrepArgs& pa) {
    // particle blocks, then sampling blocks: one per system (MH chains) or one per kBlockP samples
    if (pa.ktot > 0) nblk += pa.mh ? pa.nsys : (pa.ktot + kBlockP - 1) / kBlockP;
    if (nblk <= 0) return;
    const size_t smem = pa.mh ? (sizeof(double) + sizeof(uint32_t)) * (size_t)pa.mh_words
                              : sizeof(uint32_t) * (size_t)pa.tab_words;
    if (one)
        k_prep_f64<true><<<nblk, kBlockP, smem, st>>>(w, pos_q, fx64, cid, rank, cell_cnt, pa);
    else
        k_prep_f64<false><<<nblk, kBlockP, smem, st>>>(w, pos_q, fx64, cid, rank, cell_cnt, pa);
}

void launch_cell_assign(cudaStream_t st, bool one, const Work& w, int nblk, const uint4* fx,
                        int* cid, int* rank, int* cell_cnt, int ncell, const int* list_flag,
                        int* err) {
    if (nblk <= 0) return;
    if (one)
        k_cell_assign<true><<<nblk, kBlockP, 0, st>>>(w, fx, cid, rank, cell_cnt, ncell,
                                                      list_flag, err);
    else
        k_cell_assign<false><<<nblk, kBlockP, 0, st>>>(w, fx, cid, rank, cell_cnt, ncell,
                                                       list_flag, err);
}

void launch_scan(cudaStream_t st, int* cell_cnt, int* cell_start, int ncell, uint64_t* step_dev,
                 const uint64_t* cur_step, const int* list_flag) {
    k_scan<<<1, kScanThreads, 0, st>>>(cell_cnt, cell_start, ncell, step_dev, cur_step,
                                       list_flag);
}

void launch_scatter(cudaStream_t st, int n, const int* cid, const int* rank,
                    const int* cell_start, int* perm_tmp, const int* list_flag, int* err) {
    if (n <= 0) return;
    k_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, cid, rank, cell_start, perm_tmp, list_flag,
                                               err);
}

void launch_order(cudaStream_t st, int n, const int* cid, const int* cell_start,
                  const int* perm_tmp, const uint4* fx, uint4* spos, const double4* fx64,
                  double4* spos64, int* perm, const int* list_flag, int* iperm, int* err) {
    if (n <= 0) return;
    k_order<<<(n + 255) / 256, 256, 0, st>>>(n, cid, cell_start, perm_tmp, fx, spos, fx64, spos64,
                                             perm, list_flag, iperm, err);
}

}  // namespace rbe
