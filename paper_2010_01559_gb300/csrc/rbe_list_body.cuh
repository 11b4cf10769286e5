// rbe_list_body.cuh -- one tile of the MD step's real-space pass over the
// Verlet list (Eq. force, second term, under r_c; Eq. Ljpotential), shared by
// its own kernel (rbe_real.cu) and the fused structure-factor + list launch
// (rbe_fourier.cu).
#pragma once

#include "rbe_pair.cuh"

namespace rbe {

// The MD step's real-space pass over the list: R lanes per particle (adjacent
// lanes) take every R-th entry of the particle's list and the pair terms of
// those within the cutoffs (U gathers in flight per lane); the lanes' sums
// are added and stored per particle.  It needs nothing from the Fourier part,
// so it runs concurrently with the structure factors (and, when the list
// stands, with the no-op rebuild kernels); the Fourier-force kernel then
// completes the step.
//
// FM (forces calls): the pass runs once, after the rebuild and the Fourier
// force, and assembles per particle the total force (+ F^F), dE/dq (+ the
// Fourier part, self and background terms) and per-block FP64 partials of the
// real-space and LJ energies and virials, as the cell-scan pass does.
//
// list_body: the work of one tile (kBlockP threads, tid = the thread's index
// in them; it synchronises the block), for the pass's own kernel and for the
// fused structure-factor + list launch of the MD step.
//
// PAD: the slots of a batch past the particle's count stand for the particle
// itself (a zero displacement, which the pair terms skip) instead of being
// tested one by one: the same sums, with lanes that stay converged.  Faster
// for the pass on its own (2^20: 135 -> 122 us); inside the fused launch,
// which is issue-bound, it gains nothing, and the fused launch keeps the tests.
//
// U: list entries per lane and batch, all gathers of a batch in flight at
// once.  The pass on its own takes 4 (40 registers, more resident warps to
// hide the gathers: 2^20 122 -> 111 us); the fused launch, whose registers
// are set by its structure-factor blocks' company, takes 8.
template <int R, bool ONE, bool FM, bool PAD = true, int U = 4>
__device__ __forceinline__ void list_body(const RealArgs& a, int tile, int tid) {
    constexpr int T = kBlockP / R;               // particles per block
    const Tile tl = tile_at<ONE>(a.lw, tile);
    const int sys = tl.sys;
    const SysDev& S = sys_of<ONE>(a.lw, sys);
    const int p = tid / R, l = tid - p * R;
    const bool do_real = (a.parts & kPartReal) != 0;
    const bool do_lj = (a.parts & kPartLJ) != 0 && S.lj_eps != 0.0;
    PairConst kc;
    kc.rc2 = do_real ? S.f_rc2 : 0.f;
    kc.lj_rc2 = do_lj ? S.f_lj_rc2 : 0.f;
    kc.alpha = S.f_alpha;
    kc.sa = S.f_sqrt_alpha;
    kc.two_sa_spi = S.f_two_sa_spi;
    kc.lB = S.f_lB;
    kc.lj_s2 = S.f_lj_sigma2;
    kc.lj_eps = S.f_lj_eps;
    kc.lj_shift = S.f_lj_shift;
    kc.vir = FM && a.blk_w != nullptr;
    PairAcc acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (p < tl.count && (do_real || do_lj)) {
        const int i = tl.first + p;
        const uint4 si = a.spos[i];
        const float lbqi = kc.lB * __uint_as_float(si.w);
        const float Lu = S.L_over_2_32;
        const int* nb = a.nbr + i;
        const size_t st = (size_t)a.nbr_stride;
        // batches of U entries per lane, all gathers of a batch in flight
        // at once; the first batch is loaded alongside the count (slots within
        // the capacity always hold valid indices: the list starts zeroed).  The
        // list is read once per step: streaming loads, so that it does not
        // evict the records the gathers hit in L2.
        const int cnt = __ldcs(a.ncnt + i);
        int j[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int kk = l + q * R;
            j[q] = kk < a.nbr_cap ? __ldcs(nb + (size_t)kk * st) : (PAD ? i : 0);
        }
        if constexpr (PAD) {
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (l + q * R >= cnt) j[q] = i;
        }
        for (int k0 = l;;) {
            uint4 sj[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                if (!RBE_IN_BOUNDS(j[q], a.nbr_stride, a.err)) j[q] = i;
                sj[q] = __ldg(a.spos + j[q]);
            }
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (PAD || k0 + q * R < cnt) pair_fixed(si, sj[q], Lu, lbqi, kc, acc);
            k0 += U * R;
            if (k0 >= cnt) break;
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int kk = k0 + q * R;
                j[q] = kk < cnt ? __ldcs(nb + (size_t)kk * st) : (PAD ? i : 0);
            }
        }
    }
    float fx = acc.fx, fy = acc.fy, fz = acc.fz, ph = acc.phr;
    float ec = acc.ec, el = acc.elj, wc = acc.wc, wl = acc.wlj;
    if constexpr (R > 1) {
#pragma unroll
        for (int o = R / 2; o > 0; o >>= 1) {
            fx += __shfl_down_sync(0xffffffffu, fx, o, R);
            fy += __shfl_down_sync(0xffffffffu, fy, o, R);
            fz += __shfl_down_sync(0xffffffffu, fz, o, R);
            if constexpr (FM) {
                ph += __shfl_down_sync(0xffffffffu, ph, o, R);
                ec += __shfl_down_sync(0xffffffffu, ec, o, R);
                el += __shfl_down_sync(0xffffffffu, el, o, R);
                wc += __shfl_down_sync(0xffffffffu, wc, o, R);
                wl += __shfl_down_sync(0xffffffffu, wl, o, R);
            }
        }
        __shared__ float4 s_f[T];
        __shared__ float4 s_e[FM ? T : 1];
        if (p < tl.count && l == 0) {
            s_f[p] = make_float4(fx, fy, fz, ph);
            if constexpr (FM) s_e[p] = make_float4(ec, el, wc, wl);
        }
        __syncthreads();
        if ((int)tid < tl.count) {
            const float4 f = s_f[tid];
            fx = f.x; fy = f.y; fz = f.z; ph = f.w;
            if constexpr (FM) {
                const float4 e = s_e[tid];
                ec = e.x; el = e.y; wc = e.z; wl = e.w;
            }
        }
    }
    if constexpr (!FM) {
        // the real-space force in the caller's order, for the Fourier-force
        // kernel that adds its part and applies the thermostat
        if ((int)tid < tl.count) {
            const int o = a.perm[tl.first + tid];
            if (RBE_IN_BOUNDS(o, a.nbr_stride, a.err)) a.freal[o] = make_float4(fx, fy, fz, 0.f);
        }
    } else {
        double e_c = 0.0, e_l = 0.0, w_c = 0.0, w_l = 0.0;
        if ((int)tid < tl.count) {
            const int i = tl.first + tid;
            const int o = a.perm[i];
            float phi = ph;
            if (a.parts & kPartFourier) {
                const float4 f = a.fs[o];
                fx += f.x; fy += f.y; fz += f.z;
                if (a.phi_out) {
                    const double qi = (double)__uint_as_float(a.spos[i].w);
                    const double qs = (double)(long long)__ldcg(a.qsum_fx + sys) / kQScale;
                    phi += f.w - (float)(2.0 * S.self_coef * qi + S.bg_coef * qs);
                }
            }
            if (a.F_out) a.F_out[o] = make_float4(fx, fy, fz, 0.f);
            if (a.phi_out) a.phi_out[o] = phi;
            e_c = (double)ec;
            e_l = (double)el;
            w_c = (double)wc;
            w_l = (double)wl;
        }
        if (a.blk_e) {
            const double2 r = block_sum2_real(e_c, e_l);
            if (tid == 0) a.blk_e[tile] = r;
        }
        if (a.blk_w) {
            __syncthreads();                            // the partial buffers are reused
            const double2 r = block_sum2_real(w_c, w_l);
            if (tid == 0) a.blk_w[tile] = r;
        }
    }
}

template <int R, bool ONE, bool FM>
__global__ void __launch_bounds__(kBlockP) k_real_list(const __grid_constant__ RealArgs a) {
    if constexpr (!FM) {
        // launched twice per step: right after the prep kernel (works when the
        // list stands) and after the rebuild (works when the list was rebuilt)
        if ((*a.list_flag != 0) != (a.list_when != 0)) return;
    } else {
        if (a.flag_clear && blockIdx.x == 0 && threadIdx.x == 0) *a.flag_clear = 0;
    }
    list_body<R, ONE, FM>(a, blockIdx.x, threadIdx.x);
}

}  // namespace rbe
